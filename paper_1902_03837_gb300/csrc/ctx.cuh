// Context of libchi0 shared by its translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/chi0.h"
#include "internal.cuh"

using chi0::RhoGeom;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  bool borrowed = false;  // memory owned elsewhere (shared inputs, a batch's scratch): never freed here
};

struct chi0_ctx {
  chi0_config cfg{};
  std::vector<double> q;      // [nq][3]
  std::vector<double> om;     // [nw][2]
  int nk = 0, nb = 0, npw_max = 0;
  double a = 0.0, omega_cell = 0.0;
  cudaStream_t st = nullptr;
  std::string err;
  bool fp64 = true;

  // inputs
  std::vector<int32_t> h_npw;
  std::vector<int32_t> h_gvec;   // [nk][npw_max][3]
  std::vector<char> wf_set;
  std::vector<double> h_eps, h_occ;
  bool energies_set = false;
  DevBuf d_gvec, d_npw, d_coef, d_eps, d_occ, d_stage;

  // q-point state
  int rho_iq = -1, chi_iq = -1, eps_iq = -1;      // completed (launched) steps
  int plan_rho_iq = -1, plan_chi_iq = -1, plan_eps_iq = -1;  // planned steps
  double2* plan_eps_out = nullptr;
  // batch problems: grid_shared = the mixed grids d_U belong to another
  // problem of the same system (launch_rho then skips the wavefunction
  // transforms); group_cap > 0 limits the frequencies per operand-split pass
  bool grid_shared = false;
  int group_cap = 0;
  // band-block streaming (chi0_set_band_blocks): 0 = off.  When on, the mixed
  // grids of the m bands (occupied side) stay resident for every k (d_U), and
  // the transitions go through rho, weights and the contraction in blocks of
  // blk_nk k points x blk_nb n bands (n grids of a block in d_Ublk, its rho in
  // d_R), chi0 summed over the blocks
  int stream_nb = 0, stream_nk = 0;
  int blk_nb = 0, blk_nk = 0;
  int64_t nt_blk = 0;
  DevBuf d_Ublk;
  // Plan reuse: a plan stays valid while nothing it was made from changes.
  // plan_epoch advances whenever an input that shapes a plan changes (Miller
  // indices or sphere sizes, energies or occupations, and the settings of the
  // corrections); each plan records the epoch it was made at and the serial
  // number of the plan it builds on, so repeated steps over new coefficient
  // values skip the host set-up and its synchronisation.
  uint64_t plan_epoch = 1;
  uint64_t rho_planned_epoch = 0, chi_planned_epoch = 0, eps_planned_epoch = 0;
  uint64_t rho_plan_serial = 0, chi_plan_serial = 0;
  uint64_t chi_for_rho_serial = 0, eps_for_chi_serial = 0;
  bool capturing = false;  // inside a CUDA graph capture: no event timers
  std::vector<int32_t> h_gresp;  // [ng][3] of rho_iq
  std::vector<int32_t> h_kq, h_g0;
  std::vector<int> h_gperm;       // response indices in (Gy, Gz, Gx) order
  int n_lo = 0, Nn = 0, Nm = 0;
  int64_t nt = 0;
  RhoGeom geom{};
  DevBuf d_gresp, d_gperm, d_kq, d_g0, d_tw1, d_tw2, d_U, d_R, d_w, d_part, d_chi, d_A, d_colp, d_rowp,
      d_pinv, d_err, d_vsqrt, d_omim, d_tc;
  int nchunks = 1, kchunk = 0;
  void* tc = nullptr;  // tensor-core path state (tc.cu)
  // learned terminator (terminator.cu)
  const float* term_params = nullptr;  // device parameters; NULL = off
  int term_bf16 = 1;
  DevBuf d_termx, d_termy, d_termq, d_termw, d_termc;
  // Frequency list of the contraction: an imaginary-axis frequency is one
  // entry (real weights); a real-axis one two, the real and imaginary parts of
  // its complex weights, combined afterwards into chi0 = H_r + i H_i.
  int nwv = 0;
  bool has_real = false;
  std::vector<double> h_vval;            // [nwv] frequency value (imaginary part, or the real frequency)
  std::vector<int> h_vkind, h_vr, h_vi;  // [nwv] kind 0/1/2; [nw] entries of frequency iw (vi < 0: none)
  std::vector<int> h_vi_dev;             // the vi map as uploaded (all -1 in the mixed form: chi0 of a
                                         // real frequency comes whole from one complex contraction)
  DevBuf d_vkind, d_vr, d_vi, d_chiv;
  // Bruneval-Gonze extrapolar correction (bgterm.cu, plan in chi0_api.cu)
  int bg_on = 0;
  double bg_eps = 0.0;                 // extrapolar energy (Ha)
  int bg_nd = 0;                       // difference vectors d = G_i - G_j
  int64_t bg_ntd = 0;                  // states (k, m < Nm) with diagonal densities
  std::vector<RhoGeom> bg_geom;        // rho geometry of each chunk of the difference set
  chi0::BgChunks bg_ch{};
  DevBuf d_bgd, d_bgperm, d_bgkq, d_bgg0, d_bgrd, d_bgw, d_bgP, d_bgidx;
  // degenerate-pole grouping (Appendix B) and the double-grid frequency factor
  double grp_thresh = 0.0;             // Ha; 0: every pole its own factor
  DevBuf d_dpole;                      // [nt] pole energy of each transition's group representative
  // grouped contraction (mixed form, groups large enough to pay): the
  // frequency-independent group sums M_g = sum_{t in g} pref (f_m - f_n)
  // rho_t rho_t^H from one contraction over the transitions in group order,
  // then chi0(w) = sum_g F_g(w) M_g per frequency
  bool grouped = false;
  int ngroups = 0;                     // groups of the last grouping plan
  int64_t kgrp = 0;                    // transitions in group order, each group padded to 64
  DevBuf d_tperm;                      // [kgrp] int64 transition of each row (-1: padding)
  DevBuf d_grange;                     // [ngroups] int2 (first k-block, k-blocks) of each group
  DevBuf d_ga;                         // [nt] double pref (f_m - f_n)
  DevBuf d_gfac;                       // [nwv][ngroups] float F_g(w) of the representatives
  // sign shared by every transition weight of the imaginary-axis frequencies
  // (-1: all <= 0, +1: all >= 0, 0: mixed or not known); nonzero lets the
  // Hermitian contraction take the one-operand form chi0 = sign S S^H with
  // S = rho diag(sqrt|w|)
  int herk_sign = 0;
  int dg_nd = 0;                       // dense points per k; 0: off
  DevBuf d_epsd;                       // [nk][dg_nd][nb] dense-grid energies
  // self-energy kernel I (sigma.cu; its tensor-core operands in tc.cu):
  // rho of the quasiparticle window n in [qp_lo, qp_lo + nqp) at k and every
  // band m at k - q, W^delta and Y = W^delta conj(rho) per frequency
  RhoGeom sig_geom{};
  DevBuf d_sigR, d_sigRT, d_sigWd, d_sigY, d_sigI;
  void* sig_tc = nullptr;

  // per-stage device time: CUDA event pairs on the context's stream, summed
  // over every launch of the stage since the last chi0_get_stats
  struct Stage {
    std::vector<cudaEvent_t> ev;  // start, stop, start, stop, ...
    size_t used = 0;              // events recorded since the last readout
    double ms = 0, bytes = 0, flops = 0;
    int64_t launches = 0;
  };
  Stage stage[CHI0_NSTAGES];
  int64_t launches = 0;           // kernels launched since chi0_create
  double tc_issued_flops = 0;     // tensor-core flops issued by the last mixed contraction

  // build + Dyson in one pipeline (launch_chi0_eps): the contraction on
  // s_ct (lowest priority), the Dyson steps of finished frequencies on s_dy
  // (highest priority), both forked from and joined back into st
  cudaStream_t s_ct = nullptr, s_dy = nullptr;
  cudaStream_t s_dy2 = nullptr;      // second Dyson stream: consecutive groups alternate
  // Coefficients set from host memory on an unchanged sphere are copied on
  // s_up, one event per k point (ev_up[k], with the copy's sequence number
  // up_seq[k]), after the last wavefunction transform that read the previous
  // ones (ev_wf_done).  compute_rho then transforms the k points in chunks as
  // their copies land and starts rho on a chunk of k-pairs as soon as the
  // grids of its k and k - q points are there, so the upload overlaps rho.
  cudaStream_t s_up = nullptr;
  std::vector<cudaEvent_t> ev_up;
  std::vector<int64_t> up_seq;
  int64_t up_count = 0;
  cudaEvent_t ev_wf_done = nullptr;
  cudaEvent_t ev_join_dy2 = nullptr;
  std::vector<cudaEvent_t> ev_freq;  // [nw] contraction (and reduction) of frequency w done
  std::vector<cudaEvent_t> ev_prep;  // [nw] operand split of frequency w done
  cudaEvent_t ev_fork = nullptr, ev_join_ct = nullptr, ev_join_dy = nullptr;
};


namespace chi0 {
// record msg on c and return s
chi0_status ctx_fail(chi0_ctx* c, chi0_status s, const char* msg);
// grow b to at least bytes (device memory; contents not preserved)
chi0_status ctx_ensure(chi0_ctx* c, DevBuf& b, size_t bytes, const char* what);
// bracket the kernels of one stage on the context's stream
void stage_begin(chi0_ctx* c, int stage);
void stage_end(chi0_ctx* c, int stage, int kernels);
// split-precision tensor-core contraction (mixed mode): chi[iw][i][j] from
// R (complex64 [nt][ng]) and real weights w[iw][t]
chi0_status tc_plan(chi0_ctx* c, int64_t nt, int ng, int nw);
// ev_freq (optional, [nw]): event w is recorded once chi of frequency w is final;
// ev_prep (optional, [nw]): event w once the operand of frequency w is split
// bg (optional): the extrapolar term added to each frequency after its reduction
// vkind (optional, host, [nw]): kinds of the frequency list; an entry of kind 1
// followed by one of kind 2 is contracted once with the complex weights
// w[v] + i w[v + 1] over the full tile grid, its chi0 written at entry v
// grouped contraction: plan (operands in group order, partials per group and
// tile) and launch (splits, one contraction, the per-frequency combination)
chi0_status tc_plan_grouped(chi0_ctx* c, int ng, int nw);
chi0_status tc_launch_grouped(chi0_ctx* c, double2* chi, const cudaEvent_t* ev_freq);
// accumulate: chi += this contraction (the transitions come in blocks)
chi0_status tc_launch(chi0_ctx* c, const void* R, const double* w, int64_t nt, int ng, int nw,
                      double2* chi, const cudaEvent_t* ev_freq = nullptr,
                      const cudaEvent_t* ev_prep = nullptr, const chi0::BgApply* bg = nullptr,
                      const int* vkind = nullptr, int accumulate = 0);
void tc_release(chi0_ctx* c);
// one bounded mbarrier wait that can never be satisfied (failure detection)
cudaError_t launch_wait_probe(int* err, cudaStream_t s);
// self-energy kernel I (Eq. I_c) on the tensor cores: Y(i, t) = sum_j
// W^d_ij conj(rho_t(j)) for T transitions of the quasiparticle window, written
// in FP32 as 64 x 64 complex tiles, tile (i / 64) + (t / 64) * ceil(ng / 64)
chi0_status sig_tc_plan(chi0_ctx* c, int64_t T, int ng);
// rho of the window (the rho kernel's order ((k nqp) + a) nb + m) into the B operand
cudaError_t sig_tc_split_b(chi0_ctx* c, const float2* R, int nqp, int nb);
// W^d of one frequency from eps~^-1 (E) and V into the A operand
cudaError_t sig_tc_split_a(chi0_ctx* c, const double2* E, const double* vsqrt);
cudaError_t sig_tc_contract(chi0_ctx* c, float2* Y);
void sig_tc_release(chi0_ctx* c);
// learned terminator: network kernels and the correction of a built chi0
int mlp_nparams();
cudaError_t mlp_predict(const float* prm, const float* x, int64_t batch, int bf16, float* y,
                        cudaStream_t st);
chi0_status term_plan(chi0_ctx* c, int iq);
chi0_status term_launch(chi0_ctx* c, double2* chi);
// Batch support: a problem context that shares the inputs (coefficients,
// Miller indices, energies, occupations, dense-grid energies) of base by
// borrowing its buffers, with its own q-point state; and the scratch buffers
// of a planned context that a batch may replace by memory shared between the
// problems that run one after the other on one stream (chi0_api.cu's slots
// first, then the tensor-core state's).
chi0_ctx* make_problem_ctx(const chi0_ctx* base);
std::vector<DevBuf*> scratch_slots(chi0_ctx* c);
std::vector<DevBuf*> tc_scratch_slots(chi0_ctx* c);
// time the contraction of the first frequency for a few transition splits
// and keep the fastest (needs R and the weights of the current plan; the
// chunk-partial buffer must hold max_parts_factor times the planned partials)
chi0_status tc_tune_split(chi0_ctx* c, float* best_ms);
// plan (host set-up, allocation, uploads; may synchronise) and launch
// (kernels only, capturable) halves of compute_rho / build_chi0 / invert_eps
chi0_status plan_rho(chi0_ctx* c, int iq);
chi0_status launch_rho(chi0_ctx* c, bool with_pairs);
chi0_status plan_chi0(chi0_ctx* c, int iq);
// the weights kernel of the planned frequency list (part of launch_chi0)
chi0_status launch_weights_stage(chi0_ctx* c);
// defer_combine leaves the real-axis frequencies as their parts H_r, H_i
// (the caller combines them, frequency group by group)
chi0_status launch_chi0(chi0_ctx* c, const cudaEvent_t* ev_freq = nullptr,
                        const cudaEvent_t* ev_prep = nullptr, bool defer_combine = false);
chi0_status plan_eps(chi0_ctx* c, int iq, double2* A);
chi0_status launch_eps(chi0_ctx* c);
// build_chi0 and invert_eps as one pipeline: the Dyson step of frequency w
// overlaps the contraction of the later frequencies (mixed form without a
// terminator; otherwise the two run one after the other).  Needs plan_chi0
// and plan_eps.
// host_out (optional): a host buffer that receives eps~^-1 group by group on
// the Dyson stream; *copied tells whether it was written (only the
// overlapped pipeline does so)
chi0_status launch_chi0_eps(chi0_ctx* c, void* host_out = nullptr, bool* copied = nullptr);
}  // namespace chi0
