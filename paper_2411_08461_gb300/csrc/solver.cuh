// Mixed-precision Krylov driver on the Schur operator M_hat = A_ee - kappa^2 D_eo A_oo^-1 D_oe.
//
//   * source:        b_hat = b_e + kappa D_eo A_oo^-1 b_o            (FP64)
//   * inner solver:  BiCGStab or CGNR in the sloppy precision S with the
//                    coefficients computed on the device; check_every
//                    iterations are launched (or replayed as one CUDA graph)
//                    between host convergence checks
//   * reliable update (residual replacement, Sleijpen & van der Vorst 1996):
//                    when ||r|| < delta * max ||r|| since the last update, or
//                    at apparent convergence: x += x_s, then in FP64
//                    x_o = A_oo^-1 (b_o + kappa D_oe x_e) and the residual of the
//                    whole system b - M x; its even half (= b_hat - M_hat x_e)
//                    replaces the sloppy residual, and ||b - M x|| / ||b|| decides
//                    convergence -- so the last update is the final true-residual check.
//                    With a 16-bit inner solver the early updates (residual above a
//                    chosen 10^-k ||b||) may use the FP32 operator instead (option).
// Every (lattice, rhs) slice keeps its own coefficients and is masked out of
// every launch once it has converged.
#pragma once
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "context.cuh"

namespace wcl {

wcl_status ptc_apply(const std::vector<wcl_ctx*>& ctxs, int nrhs, const FieldRef& r, const FieldRef& z, int use_bf16);

template <int S>
struct KrylovSolver {
  static constexpr int X = (S == F64) ? F64 : F32;  // precision of the sloppy solution accumulator
  static constexpr int NMASK = 5;  // active, update, double-float, FP64, FP32 slice masks
  std::vector<wcl_ctx*> ctxs;
  wcl_ctx* c0 = nullptr;
  int nrhs = 0, nslot = 0;
  wcl_solve_params prm;
  bool cg = false;
  bool gcr = false;
  bool use_df = false;  // double-float operator for intermediate residual replacements
  bool use_s32 = false;  // FP32 operator for the early updates of a 16-bit inner solve
  double s32_level2 = 0;  // (10^-k)^2: an update above this ||r||^2 / ||b||^2 uses FP32

  FieldRef b_e, b_o, bhat, x, x_o, r64, tmp64;  // FP64
  FieldRef r, rhat, p, v, t, tmp;               // sloppy
  FieldRef xs;                                  // accumulator
  FieldRef x_df, bo_df;                         // double-float copies of x and b_o
  FieldRef x32, o32, y32, bo32;                 // FP32 work fields of the early updates
  Scalars* d_sc = nullptr;
  Scalars* h_sc = nullptr;
  int* d_active = nullptr;
  int* h_active = nullptr;
  int* d_upd = nullptr;
  int* h_upd = nullptr;
  int* d_updf = nullptr;  // slices updated with the double-float operator
  int* h_updf = nullptr;
  int* d_upd64 = nullptr;  // slices updated (or confirmed) in FP64
  int* h_upd64 = nullptr;
  int* d_upd32 = nullptr;  // slices updated with the FP32 operator
  int* h_upd32 = nullptr;
  double* d_part = nullptr;
  unsigned* d_cnt = nullptr;
  double* d_dpart = nullptr;   // dslash-epilogue partials
  unsigned* d_dcnt = nullptr;
  int dmaxch = 0;
  Batch bb;  // geometry of the BLAS / reduction launches
  int blk = 256;

  std::vector<double> stop2, r2max, b2;
  std::vector<int> iters, updates, restarts, status;

  cudaGraphExec_t gexec = nullptr;
  long long g_launches = 0, g_dslash = 0;
  size_t g_ev0 = 0, g_ev1 = 0;

  wcl_status alloc() {
    WCL_CHECK(ws_field(ctxs, "b_e", F64, nrhs, &b_e));
    WCL_CHECK(ws_field(ctxs, "b_o", F64, nrhs, &b_o));
    WCL_CHECK(ws_field(ctxs, "bhat", F64, nrhs, &bhat));
    WCL_CHECK(ws_field(ctxs, "x", F64, nrhs, &x));
    WCL_CHECK(ws_field(ctxs, "x_o", F64, nrhs, &x_o));
    WCL_CHECK(ws_field(ctxs, "r64", F64, nrhs, &r64));
    WCL_CHECK(ws_field(ctxs, "tmp64", F64, nrhs, &tmp64));
    WCL_CHECK(ws_field(ctxs, "r", S, nrhs, &r));
    WCL_CHECK(ws_field(ctxs, "rhat", S, nrhs, &rhat));
    WCL_CHECK(ws_field(ctxs, "p", S, nrhs, &p));
    WCL_CHECK(ws_field(ctxs, "v", S, nrhs, &v));
    WCL_CHECK(ws_field(ctxs, "t", S, nrhs, &t));
    WCL_CHECK(ws_field(ctxs, "tmp", S, nrhs, &tmp));
    WCL_CHECK(ws_field(ctxs, "xs", X, nrhs, &xs));
    if (use_df) {
      WCL_CHECK(ws_field(ctxs, "x_df", DF64, nrhs, &x_df));
      WCL_CHECK(ws_field(ctxs, "bo_df", DF64, nrhs, &bo_df));
    }
    if (use_s32) {
      WCL_CHECK(ws_field(ctxs, "u32_x", F32, nrhs, &x32));
      WCL_CHECK(ws_field(ctxs, "u32_o", F32, nrhs, &o32));
      WCL_CHECK(ws_field(ctxs, "u32_y", F32, nrhs, &y32));
      WCL_CHECK(ws_field(ctxs, "u32_bo", F32, nrhs, &bo32));
    }
    void* q;
    WCL_CHECK(ws_get(c0, "scalars", sizeof(Scalars) * nslot, &q));
    d_sc = static_cast<Scalars*>(q);
    WCL_CHECK(ws_get(c0, "active", sizeof(int) * NMASK * nslot, &q));
    d_active = static_cast<int*>(q);
    d_upd = d_active + nslot;
    d_updf = d_active + 2 * nslot;
    d_upd64 = d_active + 3 * nslot;
    d_upd32 = d_active + 4 * nslot;
    WCL_CHECK(ws_get(c0, "partials", sizeof(double) * nslot * RED_MAXCH * 2 * GCR_MAXK, &q));
    d_part = static_cast<double*>(q);
    WCL_CHECK(ws_get(c0, "counters", sizeof(unsigned) * nslot, &q));
    d_cnt = static_cast<unsigned*>(q);
    dmaxch = dslash_max_chunks(ctxs, S);
    WCL_CHECK(ws_get(c0, "dpartials", sizeof(double) * nslot * (size_t)dmaxch * 3, &q));
    d_dpart = static_cast<double*>(q);
    WCL_CHECK(ws_get(c0, "dcounters", sizeof(unsigned) * nslot, &q));
    d_dcnt = static_cast<unsigned*>(q);
    WCL_CHECK(hws_get(c0, "scalars", sizeof(Scalars) * nslot, &q));
    h_sc = static_cast<Scalars*>(q);
    WCL_CHECK(hws_get(c0, "active", sizeof(int) * NMASK * nslot, &q));
    h_active = static_cast<int*>(q);
    h_upd = h_active + nslot;
    h_updf = h_active + 2 * nslot;
    h_upd64 = h_active + 3 * nslot;
    h_upd32 = h_active + 4 * nslot;
    return WCL_OK;
  }

  // zero one field on every lattice
  wcl_status zero(const FieldRef& f, int prec) {
    for (size_t l = 0; l < ctxs.size(); l++) {
      const long st = ctxs[l]->lat.stride;
      size_t bytes = (size_t)nrhs * spinor_field_bytes(prec, st);
      if (prec == F16 || prec == BF16) bytes += (size_t)nrhs * st * sizeof(float);
      WCL_CUDA(cudaMemsetAsync(f.ptr[l], 0, bytes, c0->stream));
    }
    return WCL_OK;
  }

  template <int NR, typename F>
  wcl_status reduce(const F& f, const int* mask) {
    cudaError_t e = run_reduce<NR>(bb, f, mask, d_part, d_cnt, d_sc, blk, c0->stream);
    if (e != cudaSuccess) return cuda_fail(e, "reduce launch");
    count_launch(c0);
    return WCL_OK;
  }
  template <typename F>
  wcl_status map(const F& f, const int* mask) {
    cudaError_t e = run_map(bb, f, mask, blk, c0->stream);
    if (e != cudaSuccess) return cuda_fail(e, "map launch");
    count_launch(c0);
    return WCL_OK;
  }

  wcl_status sync_scalars() {
    WCL_CUDA(cudaMemcpyAsync(h_sc, d_sc, sizeof(Scalars) * nslot, cudaMemcpyDeviceToHost, c0->stream));
    WCL_CUDA(cudaStreamSynchronize(c0->stream));
    return WCL_OK;
  }
  wcl_status push_masks() {
    WCL_CUDA(cudaMemcpyAsync(d_active, h_active, sizeof(int) * NMASK * nslot, cudaMemcpyHostToDevice, c0->stream));
    return WCL_OK;
  }

  EpiSpec epi_spec;
  const EpiSpec* epi(int kind, const FieldRef& f) {
    epi_spec.kind = kind;
    epi_spec.f = f;
    epi_spec.partials = d_dpart;
    epi_spec.counters = d_dcnt;
    epi_spec.sc = d_sc;
    epi_spec.maxch = dmaxch;
    return &epi_spec;
  }

  // ---- one inner iteration (all active slices) -------------------------------
  wcl_status iteration() {
    if (!cg) {
      WCL_CHECK(map(BicgP<S>{r, p, v, d_sc}, d_active));
      WCL_CHECK(apply_mhat(ctxs, S, nrhs, v, p, tmp, false, d_active, epi(EPI_ALPHA, rhat)));  // v, alpha
      WCL_CHECK(map(BicgS<S>{r, v, d_sc}, d_active));
      WCL_CHECK(apply_mhat(ctxs, S, nrhs, t, r, tmp, false, d_active, epi(EPI_OMEGA, r)));  // t, omega
      WCL_CHECK(reduce<3>(BicgUpdate<S, X>{xs, p, r, t, rhat, d_sc}, d_active));
    } else {
      WCL_CHECK(apply_mhat(ctxs, S, nrhs, t, r, tmp, true, d_active, epi(EPI_CGZ, r)));  // z = M^+ r, beta
      WCL_CHECK(map(CgP<S>{t, p, d_sc}, d_active));
      WCL_CHECK(apply_mhat(ctxs, S, nrhs, v, p, tmp, false, d_active, epi(EPI_CGALPHA, r)));  // q = M p, alpha
      WCL_CHECK(reduce<1>(CgUpdate<S, X>{xs, p, r, v, d_sc}, d_active));
    }
    return WCL_OK;
  }

  wcl_status chunk(int n) {
    if (gexec) {
      WCL_CUDA(cudaGraphLaunch(gexec, c0->stream));
      c0->kernel_launches += g_launches;
      c0->dslash_launches += g_dslash;
      return WCL_OK;
    }
    for (int k = 0; k < n; k++) WCL_CHECK(iteration());
    return WCL_OK;
  }

  wcl_status capture(int n) {
    cudaGraph_t g = nullptr;
    WCL_CUDA(cudaStreamBeginCapture(c0->stream, cudaStreamCaptureModeThreadLocal));
    c0->capturing = true;
    c0->capture_launches = c0->capture_dslash = 0;
    g_ev0 = c0->ev_used;
    wcl_status s = WCL_OK;
    for (int k = 0; k < n && s == WCL_OK; k++) s = iteration();
    c0->capturing = false;
    cudaError_t e = cudaStreamEndCapture(c0->stream, &g);
    if (s != WCL_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    g_ev1 = c0->ev_used;
    g_launches = c0->capture_launches;
    g_dslash = c0->capture_dslash;
    e = cudaGraphInstantiate(&gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      gexec = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    return WCL_OK;
  }

  // ---- reliable update on the slices flagged in h_upd ------------------------
  // x += x_s in FP64; reconstruct x_o and evaluate the residual of the full
  // system for the current x: r_o fused into the reconstruction, r_e = b_e -
  // (A_ee x_e - kappa D_eo x_o), which equals b_hat - M_hat x_e and replaces the
  // sloppy residual.  Two operator launches per update, in `oprec`: IEEE FP64,
  // or double-float (~48-bit) for a replacement in the middle of a solve.
  wcl_status reliable_update(bool restart, int oprec, const int* mask) {
    const int bicg = (!cg && !restart) ? 1 : 0;
    if constexpr (S == F16 || S == BF16) {
      if (oprec == F32) {
        // x += x_s in FP64, then with FP32 copies: x_o = A_oo^-1 (b_o + kappa D_oe x_e),
        // (M x)_e = A_ee x_e - kappa D_eo x_o, and r = b_e - (M x)_e formed in FP64
        WCL_CHECK(map(AddInto64<X>{x, xs}, mask));
        WCL_CHECK(convert(ctxs, F32, F64, nrhs, x32, x, mask));
        WCL_CHECK(dslash(ctxs, F32, nrhs, o32, x32, &bo32, 1, false, CL_AINV, CL_NONE, C_KAPPA, C_ONE, mask));
        WCL_CHECK(dslash(ctxs, F32, nrhs, y32, o32, &x32, 0, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, mask));
        WCL_CHECK(reduce<4>(ResidualReplace<S, F32>{y32, b_e, r, rhat, FieldRef{}, bicg}, mask));
        if (restart) WCL_CHECK(restart_krylov(mask));
        return WCL_OK;
      }
    }
    if (oprec == DF64) {
      // double-float operator on double-float copies; x_o and r64 hold double-float
      // values until ResidualReplace turns r64 into the FP64 residual.  The odd
      // residual of the reconstruction (rounding level) is left to the FP64 updates.
      WCL_CHECK(map(AddInto64Split<X>{x, xs, x_df}, mask));
      WCL_CHECK(dslash(ctxs, DF64, nrhs, x_o, x_df, &bo_df, 1, false, CL_AINV, CL_NONE, C_KAPPA, C_ONE, mask));
      WCL_CHECK(dslash(ctxs, DF64, nrhs, r64, x_o, &x_df, 0, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, mask));
      WCL_CHECK(reduce<4>(ResidualReplace<S, DF64>{r64, b_e, r, rhat, FieldRef{}, bicg}, mask));
      if (restart) WCL_CHECK(restart_krylov(mask));
      return WCL_OK;
    }
    WCL_CHECK(map(AddInto64<X>{x, xs}, mask));
    WCL_CHECK(dslash_ex(ctxs, F64, nrhs, x_o, x, &b_o, &tmp64, 1, false, CL_AINV, CL_A, C_KAPPA, C_ONE, mask));
    WCL_CHECK(dslash(ctxs, F64, nrhs, r64, x_o, &x, 0, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, mask));
    WCL_CHECK(reduce<4>(ResidualReplace<S, F64>{r64, b_e, r, rhat, tmp64, bicg}, mask));
    if (restart) WCL_CHECK(restart_krylov(mask));
    return WCL_OK;
  }

  // The updates of one check point for the slices in h_upd.  A slice that may
  // finish (it looks converged, hit maxiter, broke down or went non-finite) is
  // evaluated in IEEE FP64; the others use the double-float operator, and any of
  // those that then meets the tolerance is re-evaluated in FP64.  So every
  // status and every reported true residual comes from an FP64 evaluation.
  // On return h_upd64[s] marks the slices whose aux[] holds an FP64 result.
  wcl_status update_round(bool restart) {
    bool any_df = false, any_64 = false, any_32 = false;
    for (int s = 0; s < nslot; s++) {
      h_updf[s] = h_upd64[s] = h_upd32[s] = 0;
      if (!h_upd[s]) continue;
      const double r2 = h_sc[s].r2;
      const bool ending = r2 <= stop2[s] || iters[s] >= prm.maxiter || (h_sc[s].flags & 1) || !(r2 == r2) ||
                          !use_df;
      if (ending) {
        h_upd64[s] = 1;
        any_64 = true;
      } else if (use_s32 && r2 > s32_level2 * b2[s]) {
        h_upd32[s] = 1;
        any_32 = true;
      } else {
        h_updf[s] = 1;
        any_df = true;
      }
    }
    WCL_CHECK(push_masks());
    if (any_32) WCL_CHECK(reliable_update(restart, F32, d_upd32));
    if (any_df) WCL_CHECK(reliable_update(restart, DF64, d_updf));
    if (any_64) WCL_CHECK(reliable_update(restart, F64, d_upd64));
    WCL_CHECK(sync_scalars());
    profile_sync();
    bool confirm = false;
    for (int s = 0; s < nslot; s++) {
      if (!h_updf[s]) continue;
      const double tr2 = h_sc[s].aux[3];
      h_updf[s] = 0;
      if (tr2 <= stop2[s] || !(tr2 == tr2)) {
        h_upd64[s] = 2;  // confirm in FP64
        confirm = true;
      }
    }
    if (confirm) {
      for (int s = 0; s < nslot; s++) h_updf[s] = (h_upd64[s] == 2);
      WCL_CHECK(push_masks());
      WCL_CHECK(reliable_update(restart, F64, d_updf));
      WCL_CHECK(sync_scalars());
      profile_sync();
      for (int s = 0; s < nslot; s++) h_updf[s] = 0;
    }
    for (int s = 0; s < nslot; s++) h_upd32[s] = 0;
    return WCL_OK;
  }

  // fresh Krylov space from the current residual on the flagged slices
  wcl_status restart_krylov(const int* mask) {
    if (!cg) {
      WCL_CHECK(convert(ctxs, S, S, nrhs, rhat, r, mask));
      WCL_CHECK(map(ZeroPair<S>{p, v}, mask));
      WCL_CHECK(reduce<3>(BicgRho<S>{rhat, r, RHO_INIT}, mask));
    } else {
      WCL_CHECK(map(ZeroPair<S>{p, v}, mask));
      WCL_CHECK(map(ResetCg{d_sc}, mask));
    }
    return WCL_OK;
  }

  void profile_sync() {
    if (!c0->profiling) return;
    if (gexec) {
      profile_accum_range(c0, g_ev0, g_ev1);
      profile_flush(c0, g_ev1);
    } else {
      profile_flush(c0, 0);
    }
  }

  // ---- flexible GCR on M_hat (restarted every m steps) ------------------------
  // z_k = N(r) (the learned network, or z_k = r for plain GCR), w_k = M_hat z_k,
  // w_k and z_k orthogonalised against W by classical Gram-Schmidt applied twice
  // (as stable as modified Gram-Schmidt, two passes instead of k), then
  // alpha = <w_k, r>/||w_k||^2, x += alpha z_k, r -= alpha w_k, and w_k, z_k
  // rescaled to unit ||w_k||.  Every restart is a reliable update.
  wcl_status loop_gcr(int& nactive, bool learned, bool mgb = false) {
    const int m = std::min(std::max(1, prm.gcr_nkrylov), GCR_MAXK);
    FieldRef Z{}, W{}, r32{}, z32{};
    long vstride[MAXLAT] = {}, nvstride[MAXLAT] = {};
    const bool half = (S == F16 || S == BF16);
    for (size_t l = 0; l < ctxs.size(); l++) {
      wcl_ctx* c = ctxs[l];
      const long st = c->lat.stride;
      const size_t chunk = (size_t)nrhs * spinor_field_bytes(S, st);
      const size_t nb = half ? (size_t)nrhs * st * sizeof(float) : 0;
      const size_t blockb = (chunk + nb + 255) / 256 * 256;
      void *pz, *pw;
      WCL_CHECK(ws_get(c, "gcr_Z" + std::to_string(S), blockb * m, &pz));
      WCL_CHECK(ws_get(c, "gcr_W" + std::to_string(S), blockb * m, &pw));
      Z.ptr[l] = pz;
      W.ptr[l] = pw;
      Z.norm[l] = half ? reinterpret_cast<float*>(static_cast<char*>(pz) + chunk) : nullptr;
      W.norm[l] = half ? reinterpret_cast<float*>(static_cast<char*>(pw) + chunk) : nullptr;
      vstride[l] = (long)blockb;
      nvstride[l] = (long)(blockb / sizeof(float));
    }
    auto vec = [&](const FieldRef& base, int j) {
      FieldRef f{};
      for (size_t l = 0; l < ctxs.size(); l++) {
        f.ptr[l] = static_cast<char*>(base.ptr[l]) + (size_t)j * vstride[l];
        f.norm[l] = base.norm[l] ? base.norm[l] + (size_t)j * nvstride[l] : nullptr;
      }
      return f;
    };
    if (learned && S != F32) {
      WCL_CHECK(ws_field(ctxs, "gcr_r32", F32, nrhs, &r32));
      WCL_CHECK(ws_field(ctxs, "gcr_z32", F32, nrhs, &z32));
    }
    void* q;
    WCL_CHECK(ws_get(c0, "gcr_betas", sizeof(double2) * nslot * GCR_MAXK, &q));
    double2* betas = static_cast<double2*>(q);
    const double d2 = prm.delta_reliable * prm.delta_reliable;
    int k = 0;
    while (nactive > 0) {
      const FieldRef Zk = vec(Z, k), Wk = vec(W, k);
      if (mgb) {
        WCL_CHECK(mg_batched_cycle(c0, nrhs, r.ptr[0], Zk.ptr[0]));
      } else if (learned) {
        if (S == F32) {
          WCL_CHECK(ptc_apply(ctxs, nrhs, r, Zk, 1));
        } else {
          WCL_CHECK(convert(ctxs, F32, S, nrhs, r32, r, d_active));
          WCL_CHECK(ptc_apply(ctxs, nrhs, r32, z32, 1));
          WCL_CHECK(convert(ctxs, S, F32, nrhs, Zk, z32, d_active));
        }
      } else {
        WCL_CHECK(convert(ctxs, S, S, nrhs, Zk, r, d_active));
      }
      WCL_CHECK(apply_mhat(ctxs, S, nrhs, Wk, Zk, tmp, false, d_active));
      for (int pass = 0; pass < 2 && k > 0; pass++) {
        GcrMultiDot<S> md{};
        md.W = W;
        md.w = Wk;
        md.k = k;
        md.betas = betas;
        md.sc_base = d_sc;
        GcrMultiAxpy<S> ma{};
        ma.W = W;
        ma.Z = Z;
        ma.w = Wk;
        ma.z = Zk;
        ma.k = k;
        ma.betas = betas;
        for (size_t l = 0; l < ctxs.size(); l++) {
          md.vstride[l] = ma.vstride[l] = vstride[l];
          md.nvstride[l] = ma.nvstride[l] = nvstride[l];
        }
        WCL_CHECK(reduce<2 * GCR_MAXK>(md, d_active));
        WCL_CHECK(map(ma, d_active));
      }
      WCL_CHECK(reduce<3>(GcrAlpha<S>{Wk, r}, d_active));
      WCL_CHECK(reduce<1>(GcrUpdate<S, X>{xs, r, Wk, Zk, d_sc}, d_active));
      k++;
      WCL_CHECK(sync_scalars());
      profile_sync();
      bool any = false;
      for (int s = 0; s < nslot; s++) {
        h_upd[s] = 0;
        if (!h_active[s]) continue;
        iters[s] += 1;
        const double r2 = h_sc[s].r2;
        r2max[s] = std::max(r2max[s], r2);
        const bool brk = (h_sc[s].flags & 1) || !(r2 == r2);
        if (k == m || r2 <= stop2[s] || r2 < d2 * r2max[s] || brk || iters[s] >= prm.maxiter) any = true;
      }
      if (!any) continue;
      for (int s = 0; s < nslot; s++) h_upd[s] = h_active[s];
      WCL_CHECK(update_round(false));
      for (int s = 0; s < nslot; s++) {
        if (!h_upd[s]) continue;
        updates[s]++;
        const double tr2 = h_sc[s].aux[3];
        r2max[s] = h_sc[s].aux[0];
        if (!h_upd64[s]) {
          h_sc[s].flags = 0;
          continue;  // double-float replacement only: keep iterating
        }
        if (!(tr2 == tr2) || std::isinf(tr2)) {
          status[s] = WCL_ERR_NONFINITE;
          h_active[s] = 0;
          nactive--;
        } else if (tr2 <= stop2[s]) {
          h_active[s] = 0;
          nactive--;
        } else if (iters[s] >= prm.maxiter) {
          status[s] = WCL_ERR_NOT_CONVERGED;
          h_active[s] = 0;
          nactive--;
        } else if (h_sc[s].flags & 1) {
          if (++restarts[s] > 3) {
            status[s] = WCL_ERR_BREAKDOWN;
            h_active[s] = 0;
            nactive--;
          }
        }
        h_sc[s].flags = 0;
      }
      for (int s = 0; s < nslot; s++) h_upd[s] = 0;
      WCL_CUDA(cudaMemcpyAsync(d_sc, h_sc, sizeof(Scalars) * nslot, cudaMemcpyHostToDevice, c0->stream));
      WCL_CHECK(push_masks());
      k = 0;  // restart from the replaced residual
    }
    return WCL_OK;
  }

  // ---- the whole solve -------------------------------------------------------
  wcl_status run(const SolveIO& io, wcl_solve_info* info) {
    auto t0 = std::chrono::steady_clock::now();
    c0 = ctxs[0];
    nslot = (int)ctxs.size() * nrhs;
    gcr = prm.solver == WCL_FGCR_LEARNED || prm.solver == WCL_GCR || prm.solver == WCL_FGCR_MG_BATCHED;
    cg = prm.solver == WCL_CGNR || gcr;  // GCR residual replacement keeps no BiCGStab state
    blk = c0->blas_block;
    bb = make_batch(ctxs, nrhs, blk, RED_MAXCH);
    // Intermediate residual replacements of a mixed-precision solve use the
    // double-float operator (FP32 pipes); every final one is IEEE FP64.
    use_df = S != F64 && prm.outer == WCL_DF64;
    use_s32 = (S == F16 || S == BF16) && use_df && c0->sloppy_updates > 0 && !gcr;
    if (use_s32) s32_level2 = std::pow(10.0, -2.0 * c0->sloppy_updates);
    WCL_CHECK(alloc());
    stop2.assign(nslot, 0);
    b2.assign(nslot, 0);
    r2max.assign(nslot, 0);
    iters.assign(nslot, 0);
    updates.assign(nslot, 0);
    restarts.assign(nslot, 0);
    status.assign(nslot, WCL_OK);
    WCL_CUDA(cudaMemsetAsync(d_sc, 0, sizeof(Scalars) * nslot, c0->stream));
    for (int s = 0; s < nslot; s++) h_active[s] = 1, h_upd[s] = h_updf[s] = h_upd64[s] = h_upd32[s] = 0;
    WCL_CHECK(push_masks());
    WCL_CUDA(cudaMemsetAsync(c0->d_flags, 0, sizeof(int), c0->stream));

    // import b (both parities) into FP64 internal fields
    for (size_t l = 0; l < ctxs.size(); l++) {
      const LatticeDevice& L = ctxs[l]->lat;
      const long rs = 2 * L.vh * 12;
      WCL_CUDA(import_fermion(L, io.d_b[l], rs, 0, nrhs, b_e.ptr[l], c0->d_flags, c0->stream));
      WCL_CUDA(import_fermion(L, io.d_b[l], rs, L.vh * 12, nrhs, b_o.ptr[l], c0->d_flags, c0->stream));
      count_launch(c0);
      count_launch(c0);
    }
    // b_hat = b_e + kappa D_eo A_oo^-1 b_o
    // In a mixed-precision solve b_hat only seeds the iteration: the first
    // residual replacement evaluates b_e - (M x)_e from b itself, with x_o
    // rebuilt from b_o, so every later residual and every reported one is
    // independent of how b_hat was rounded.  It is therefore formed with the
    // sloppy operator (v, t, tmp and r are free until the first iteration).
    if (use_df) WCL_CHECK(convert(ctxs, DF64, F64, nrhs, bo_df, b_o, nullptr));
    if (use_s32) WCL_CHECK(convert(ctxs, F32, F64, nrhs, bo32, b_o, nullptr));
    if (S != F64) {
      WCL_CHECK(convert(ctxs, S, F64, nrhs, v, b_o, nullptr));
      WCL_CHECK(convert(ctxs, S, F64, nrhs, t, b_e, nullptr));
      WCL_CHECK(clover_apply(ctxs, S, nrhs, tmp, v, 1, CL_AINV, nullptr));
      WCL_CHECK(dslash(ctxs, S, nrhs, r, tmp, &t, 0, false, CL_NONE, CL_NONE, C_KAPPA, C_ONE, nullptr));
      WCL_CHECK(convert(ctxs, F64, S, nrhs, bhat, r, nullptr));
    } else {
      WCL_CHECK(clover_apply(ctxs, F64, nrhs, tmp64, b_o, 1, CL_AINV, nullptr));
      WCL_CHECK(dslash(ctxs, F64, nrhs, bhat, tmp64, &b_e, 0, false, CL_NONE, CL_NONE, C_KAPPA, C_ONE, nullptr));
    }
    WCL_CHECK(reduce<1>(Norm2<F64>{b_e, b_e, 2, 0, 0}, nullptr));
    WCL_CHECK(reduce<1>(Norm2<F64>{b_o, b_o, 2, 1, 0}, nullptr));
    WCL_CHECK(reduce<1>(Norm2<F64>{bhat, bhat, 1, 0, 0}, nullptr));
    WCL_CHECK(zero(x, F64));
    WCL_CHECK(zero(x_o, F64));
    WCL_CHECK(zero(xs, X));
    WCL_CHECK(zero(p, S));
    WCL_CHECK(zero(v, S));
    WCL_CHECK(convert(ctxs, S, F64, nrhs, r, bhat, nullptr));
    WCL_CHECK(convert(ctxs, S, S, nrhs, rhat, r, nullptr));
    if (!cg) WCL_CHECK(reduce<3>(BicgRho<S>{rhat, r, RHO_INIT}, nullptr));
    WCL_CHECK(sync_scalars());
    int hflag = 0;
    WCL_CUDA(cudaMemcpy(&hflag, c0->d_flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (hflag & 1) {
      set_error("non-finite entry in the right-hand side");
      return WCL_ERR_NONFINITE;
    }
    const double tol2 = prm.tol * prm.tol;
    const double safety = 0.81;  // aim 10% below the target on the Schur residual
    int nactive = 0;
    for (int s = 0; s < nslot; s++) {
      const double bb = h_sc[s].aux[2];
      b2[s] = bb;
      stop2[s] = tol2 * bb * safety;
      r2max[s] = h_sc[s].aux[1];
      if (!(bb > 0.0)) {
        h_active[s] = 0;  // zero source: x = 0 exactly
      } else {
        nactive++;
      }
    }
    WCL_CHECK(push_masks());

    const int ce = std::max(1, prm.check_every);
    const double d2 = prm.delta_reliable * prm.delta_reliable;
    if (gcr) WCL_CHECK(loop_gcr(nactive, prm.solver == WCL_FGCR_LEARNED, prm.solver == WCL_FGCR_MG_BATCHED));
    // events inside captured graphs cannot be timed: profiling launches directly
    bool graphs = prm.use_graphs != 0 && !c0->profiling;
    if (graphs && !gcr) {
      // let the tuner see the operator launches of the loop before they are captured
      // (p is zero and v, t, tmp are overwritten by the first iteration)
      WCL_CHECK(apply_mhat(ctxs, S, nrhs, v, p, tmp, false, d_active));
      if (cg) WCL_CHECK(apply_mhat(ctxs, S, nrhs, v, p, tmp, true, d_active));
    }
    while (nactive > 0) {
      if (graphs && !gexec) {
        wcl_status s = capture(ce);
        if (s != WCL_OK) {
          graphs = false;  // fall back to direct launches of the same kernels
          set_error("");
        }
      }
      WCL_CHECK(chunk(ce));
      WCL_CHECK(sync_scalars());
      profile_sync();
      bool any = false;
      for (int s = 0; s < nslot; s++) {
        h_upd[s] = 0;
        if (!h_active[s]) continue;
        iters[s] += ce;
        const double r2 = h_sc[s].r2;
        r2max[s] = std::max(r2max[s], r2);
        const bool brk = (h_sc[s].flags & 1) || !(r2 == r2);
        if (r2 <= stop2[s] || r2 < d2 * r2max[s] || brk || iters[s] >= prm.maxiter) {
          h_upd[s] = 1;
          any = true;
        }
      }
      if (!any) continue;
      WCL_CHECK(update_round(prm.restart_on_update != 0));
      bool restart_any = false;
      for (int s = 0; s < nslot; s++) {
        if (!h_upd[s]) continue;
        updates[s]++;
        const double tr2 = h_sc[s].aux[3];  // full-system true residual^2
        const bool brk = (h_sc[s].flags & 1) != 0;
        r2max[s] = h_sc[s].aux[0];
        if (!h_upd64[s]) {
          h_upd[s] = 0;  // double-float replacement only: keep iterating
          continue;
        }
        if (!(tr2 == tr2) || std::isinf(tr2)) {
          status[s] = WCL_ERR_NONFINITE;
          h_active[s] = 0;
          nactive--;
        } else if (tr2 <= stop2[s]) {
          h_active[s] = 0;
          nactive--;
        } else if (iters[s] >= prm.maxiter) {
          status[s] = WCL_ERR_NOT_CONVERGED;
          h_active[s] = 0;
          nactive--;
        } else if (brk) {
          if (++restarts[s] > 3) {
            status[s] = WCL_ERR_BREAKDOWN;
            h_active[s] = 0;
            nactive--;
          } else {
            restart_any = true;
          }
        }
        if (!(brk && h_active[s])) h_upd[s] = 0;  // keep the mask only for restarts
      }
      if (restart_any) {
        for (int s = 0; s < nslot; s++) h_sc[s].flags = 0;
        WCL_CHECK(push_masks());
        WCL_CUDA(cudaMemcpyAsync(d_sc, h_sc, sizeof(Scalars) * nslot, cudaMemcpyHostToDevice, c0->stream));
        WCL_CHECK(restart_krylov(d_upd));
      }
      for (int s = 0; s < nslot; s++) h_upd[s] = 0;
      WCL_CHECK(push_masks());
    }
    if (gexec) {
      cudaGraphExecDestroy(gexec);
      gexec = nullptr;
    }

    // finish: every right-hand side ended on a reliable update, which folded
    // x_s into x, reconstructed x_o and left ||b - M x||^2 in aux[3]
    for (size_t l = 0; l < ctxs.size(); l++) {
      const LatticeDevice& L = ctxs[l]->lat;
      const long rs = 2 * L.vh * 12;
      WCL_CUDA(export_fermion(L, x.ptr[l], nrhs, io.d_x[l], rs, 0, c0->stream));
      WCL_CUDA(export_fermion(L, x_o.ptr[l], nrhs, io.d_x[l], rs, L.vh * 12, c0->stream));
      count_launch(c0);
      count_launch(c0);
    }
    WCL_CHECK(sync_scalars());
    profile_flush(c0, 0);
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    wcl_status worst = WCL_OK;
    for (int s = 0; s < nslot; s++) {
      const double b2 = h_sc[s].aux[2];
      const double tr = b2 > 0 ? std::sqrt(h_sc[s].aux[3] / b2) : 0.0;
      info[s].iters = iters[s];
      info[s].true_residual = tr;
      info[s].reliable_updates = updates[s];
      if (status[s] == WCL_OK && !(tr <= prm.tol)) status[s] = (tr == tr) ? WCL_ERR_NOT_CONVERGED : WCL_ERR_NONFINITE;
      info[s].status = status[s];
      info[s].seconds = secs;
      if (worst == WCL_OK && status[s] != WCL_OK) worst = (wcl_status)status[s];
    }
    if (worst != WCL_OK) set_error("right-hand side did not reach the tolerance: %s", worst == WCL_ERR_NOT_CONVERGED ? "maxiter" : "breakdown / non-finite");
    return worst;
  }
};

template <int S>
wcl_status krylov_solve(const std::vector<wcl_ctx*>& ctxs, int nrhs, const wcl_solve_params& prm, const SolveIO& io,
                        wcl_solve_info* info) {
  KrylovSolver<S> ks;
  ks.ctxs = ctxs;
  ks.nrhs = nrhs;
  ks.prm = prm;
  wcl_status st = ks.run(io, info);
  if (ks.gexec) cudaGraphExecDestroy(ks.gexec);
  return st;
}

}  // namespace wcl
