// Context helpers: errors, workspace, batch geometry, operator launches, profiling.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "context.cuh"

namespace wcl {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
const char* last_error_text() { return g_err; }

wcl_status cuda_fail(cudaError_t e, const char* where) {
  set_error("%s: %s", where, cudaGetErrorString(e));
  cudaGetLastError();  // clear a sticky-free error so later calls can proceed
  return e == cudaErrorMemoryAllocation ? WCL_ERR_OOM : WCL_ERR_CUDA;
}

wcl_status ws_get(wcl_ctx* c, const std::string& name, size_t bytes, void** out) {
  auto& b = c->ws[name];
  if (b.bytes < bytes) {
    if (c->capturing) {
      set_error("workspace %s requested during graph capture", name.c_str());
      return WCL_ERR_INVALID_ARG;
    }
    if (b.p) {
      WCL_CUDA(cudaStreamSynchronize(c->stream));
      WCL_CUDA(cudaFree(b.p));
      b.p = nullptr;
      b.bytes = 0;
    }
    WCL_CUDA(cudaMalloc(&b.p, bytes));
    WCL_CUDA(cudaMemsetAsync(b.p, 0, bytes, c->stream));
    b.bytes = bytes;
  }
  *out = b.p;
  return WCL_OK;
}

wcl_status ws_field(const std::vector<wcl_ctx*>& ctxs, const std::string& name, int prec, int nrhs, FieldRef* out) {
  memset(out, 0, sizeof(*out));
  for (size_t l = 0; l < ctxs.size(); l++) {
    wcl_ctx* c = ctxs[l];
    const long st = c->lat.stride;
    size_t bytes = (size_t)nrhs * spinor_field_bytes(prec, st);
    const size_t nbytes = (prec == F16 || prec == BF16) ? (size_t)nrhs * st * sizeof(float) : 0;
    void* p = nullptr;
    WCL_CHECK(ws_get(c, name + "#" + std::to_string(prec), bytes + nbytes, &p));
    out->ptr[l] = p;
    out->norm[l] = nbytes ? reinterpret_cast<float*>(static_cast<char*>(p) + bytes) : nullptr;
  }
  return WCL_OK;
}

Batch make_batch(const std::vector<wcl_ctx*>& ctxs, int nrhs, int block, int cap) {
  Batch b;
  memset(&b, 0, sizeof b);
  b.nlat = (int)ctxs.size();
  int blocks = 0;
  for (int l = 0; l < b.nlat; l++) {
    const LatticeDevice& L = ctxs[l]->lat;
    LatGeom& g = b.lat[l];
    for (int d = 0; d < 4; d++) g.dims[d] = L.dims[d];
    g.lxh = L.dims[0] / 2;
    g.vh = (int)L.vh;
    g.stride = L.stride;
    g.nrhs = nrhs;
    long nch = (L.vh + block - 1) / block;
    if (cap > 0 && nch > cap) nch = cap;
    g.nchunk = (int)nch;
    g.block_begin = blocks;
    g.slot_base = l * nrhs;
    g.tb = (float)L.tb;
    g.tw = L.tw;
    g.tw_f = (float)L.tw;
    g.tbw_f = (float)((double)L.tb * L.tw);
    blocks += g.nchunk * nrhs;
  }
  b.total_blocks = blocks;
  return b;
}

static void spinor_site_bytes(int prec, double& sp, double& link, double& clov) {
  switch (prec) {
    case F64:
    case DF64: sp = 192; link = 144; clov = 576; break;
    case F32: sp = 96; link = 48; clov = 288; break;
    default: sp = 52; link = 24; clov = 148; break;
  }
}

static wcl_ctx::Timed* prof_begin(wcl_ctx* c) {
  if (!c->profiling) return nullptr;
  if (c->ev_used == c->ev_pool.size()) {
    wcl_ctx::Timed t;
    if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(t);
  }
  wcl_ctx::Timed* t = &c->ev_pool[c->ev_used++];
  cudaEventRecord(t->a, c->stream);
  return t;
}

wcl_status dslash(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const FieldRef& out, const FieldRef& in,
                  const FieldRef* x, int out_parity, bool dagger, CloverSel post, CloverSel pre, Coef alpha,
                  Coef beta, const int* active) {
  return dslash_ex(ctxs, prec, nrhs, out, in, x, nullptr, out_parity, dagger, post, pre, alpha, beta, active);
}

bool use_tc(const wcl_ctx* c, int prec, int nrhs, int mode) {
  return c->tensor_cores && prec == F16 && nrhs >= 4 && nrhs <= 16 &&
         (mode == MODE_POST || mode == (MODE_XPAY | MODE_PRE));
}

bool use_mrhs(const wcl_ctx* c, int prec, int nrhs, int mode) {
  return c->shared_links && prec != DF64 && nrhs >= 4 && nrhs <= 16 &&
         (mode == MODE_POST || mode == (MODE_XPAY | MODE_PRE));
}

bool use_pair(const wcl_ctx* c, int prec, int nrhs, int mode) {
  return use_mrhs(c, prec, nrhs, mode) && (prec == F32 || prec == F16 || prec == BF16);
}

int dslash_max_chunks(const std::vector<wcl_ctx*>& ctxs, int prec) {
  // smallest site tile any dslash variant may use, so that the partials fit every variant
  (void)prec;
  const int block = std::min(kTuneMinBlock, std::min(tc_tile_sites(), MR_SITES));
  long m = 1;
  for (auto* c : ctxs) m = std::max(m, (c->lat.vh + block - 1) / block);
  return (int)m;
}

// z planes per block of the multi-RHS kernel's tile order: the largest divisor of
// Lz keeping Ly * zblk * (tiles per row) <= 512 tiles between a site and its t
// neighbours; 0 (site order) when tiles are not whole parts of x rows or the lattice
// is small enough for site order to keep them in L2 anyway
static int mrhs_zblock(const LatGeom& g, int ts) {
  if (g.lxh % ts != 0) return 0;
  const long tpr = g.lxh / ts, Ly = g.dims[1], Lz = g.dims[2];
  if (Ly * Lz * tpr <= 512) return 0;
  for (int bz = Lz; bz >= 1; bz--)
    if (Lz % bz == 0 && Ly * bz * tpr <= 512) return bz;
  return 1;
}

// ---------------------------------------------------------------------------
// Kernel variants of one dslash configuration and their launch.
static cudaError_t launch_variant(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, DslashArgs a, bool dagger,
                                  int mode, TuneChoice ch, cudaStream_t st) {
  if (ch.variant == V_THREAD) {
    a.b = make_batch(ctxs, nrhs, ch.block, 0);
    switch (prec) {
      case F64: return launch_dslash<F64>(a, dagger, mode, ch.block, st);
      case DF64: return launch_dslash<DF64>(a, dagger, mode, ch.block, st);
      case F32: return launch_dslash<F32>(a, dagger, mode, ch.block, st);
      case F16: return launch_dslash<F16>(a, dagger, mode, ch.block, st);
      default: return launch_dslash<BF16>(a, dagger, mode, ch.block, st);
    }
  }
  // one CTA covers all right-hand sides of its sites
  const int ts = ch.variant == V_TC ? tc_tile_sites() : ch.block;
  a.b = make_batch(ctxs, 1, ts, 0);
  for (size_t l = 0; l < ctxs.size(); l++) {
    a.b.lat[l].slot_base = (int)l * nrhs;
    if (ch.variant == V_SMEM_ZB || ch.variant == V_PAIR_ZB || ch.variant == V_SMEM_PF_ZB)
      a.b.lat[l].zblk = mrhs_zblock(a.b.lat[l], ts);
  }
  a.nrhs_tc = nrhs;
  if (ch.variant == V_TC) return launch_dslash_tc(prec, a, dagger, mode, st);
  if (ch.variant == V_TMA || ch.variant == V_TMA_TILE) {
    if (prec != F32) return cudaErrorInvalidValue;
    ctxs[0]->wait_check = true;
    return launch_dslash_tma(a, dagger, mode, st, ctxs[0]->d_flags, ch.variant == V_TMA);
  }
  if (ch.variant == V_PAIR || ch.variant == V_PAIR_ZB) {
    switch (prec) {
      case F32: return launch_dslash_pair<F32>(a, dagger, mode, ts, st);
      case F16: return launch_dslash_pair<F16>(a, dagger, mode, ts, st);
      case BF16: return launch_dslash_pair<BF16>(a, dagger, mode, ts, st);
      default: return cudaErrorInvalidValue;
    }
  }
  const bool async = ch.variant == V_SMEM_ASYNC;
  const bool pf = ch.variant == V_SMEM_PF || ch.variant == V_SMEM_PF_ZB;
  switch (prec) {
    case F64: return launch_dslash_mrhs<F64>(a, dagger, mode, ts, st, async, pf);
    case F32: return launch_dslash_mrhs<F32>(a, dagger, mode, ts, st, async, pf);
    case F16: return launch_dslash_mrhs<F16>(a, dagger, mode, ts, st, async, pf);
    default: return launch_dslash_mrhs<BF16>(a, dagger, mode, ts, st, async, pf);
  }
}

static bool same_ptr(const FieldRef& w, const FieldRef& r, int nlat) {
  for (int l = 0; l < nlat; l++)
    if (w.ptr[l] && w.ptr[l] == r.ptr[l]) return true;
  return false;
}

// Pick the variant for this configuration: from the cache, else by timing every
// candidate (without the fused reduction, whose result must be produced once).
static TuneChoice choose_variant(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const DslashArgs& a,
                                 bool dagger, int mode) {
  wcl_ctx* c0 = ctxs[0];
  const int nlat = (int)ctxs.size();
  const bool tc_ok = use_tc(c0, prec, nrhs, mode);
  const bool mr_ok = use_mrhs(c0, prec, nrhs, mode);
  const bool pair_ok = use_pair(c0, prec, nrhs, mode);
  bool tma_ok = mr_ok && prec == F32 && nlat == 1;
  if (tma_ok) {
    LatGeom gg{};
    gg.lxh = c0->lat.dims[0] / 2;
    gg.vh = (int)c0->lat.vh;
    tma_ok = tma_eligible(gg, nrhs);
  }
  TuneChoice dflt{V_THREAD, c0->dslash_block[prec == DF64 ? F64 : prec]};
  if (tc_ok)
    dflt = {V_TC, tc_tile_sites()};
  else if (tma_ok && c0->tma_staging)
    dflt = {c0->tma_staging == 2 ? V_TMA_TILE : V_TMA, 16};
  else if (pair_ok && c0->paired_rhs)
    dflt = c0->blocked_tiles ? TuneChoice{V_PAIR_ZB, 16} : TuneChoice{V_PAIR, c0->shared_links};
  else if (mr_ok && c0->staged_spinors && prec != F64)
    dflt = {V_SMEM_ASYNC, 16};
  else if (mr_ok && c0->prefetch_spinors && prec != F64)
    dflt = c0->blocked_tiles ? TuneChoice{V_SMEM_PF_ZB, 16} : TuneChoice{V_SMEM_PF, 16};
  else if (mr_ok && c0->blocked_tiles)
    dflt = {V_SMEM_ZB, 16};
  else if (mr_ok)
    dflt = {V_SMEM, prec == F64 ? 16 : c0->shared_links};
  std::string key = "dslash p" + std::to_string(prec) + " m" + std::to_string(mode) + " d" + std::to_string(dagger) +
                    " n" + std::to_string(nrhs) + " o" + std::to_string((int)tc_ok) + std::to_string((int)mr_ok) +
                    std::to_string((int)c0->staged_spinors) + std::to_string((int)c0->blocked_tiles) +
                    std::to_string((int)c0->paired_rhs) + std::to_string((int)c0->prefetch_spinors) +
                    std::to_string((int)c0->tma_staging);
  for (auto* c : ctxs)
    key += " " + std::to_string(c->lat.dims[0]) + "x" + std::to_string(c->lat.dims[1]) + "x" +
           std::to_string(c->lat.dims[2]) + "x" + std::to_string(c->lat.dims[3]);
  TuneChoice ch;
  if (tune_lookup(key, &ch)) return ch;
  // only time when the launches may be repeated: outside graph capture, outputs not read
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c0->stream, &cs);
  if (!c0->autotune || c0->capturing || cs != cudaStreamCaptureStatusNone || same_ptr(a.out, a.in, nlat) ||
      same_ptr(a.out, a.x, nlat) || same_ptr(a.out, a.f, nlat) || same_ptr(a.out2, a.in, nlat) ||
      same_ptr(a.out2, a.x, nlat) || same_ptr(a.out2, a.f, nlat))
    return dflt;
  std::vector<TuneChoice> cand;
  for (int blk : {64, 128, 256, 512}) cand.push_back({V_THREAD, blk});
  if (mr_ok) {
    cand.push_back({V_SMEM, 8});
    cand.push_back({V_SMEM, 16});
    if (prec != F64) {
      cand.push_back({V_SMEM, 32});  // FP64 32-site tiles exceed 48 KB of static shared memory
      cand.push_back({V_SMEM_ASYNC, 16});
      cand.push_back({V_SMEM_PF, 16});
    }
    bool zb = false;
    for (auto* c : ctxs) {
      LatGeom gg{};
      gg.lxh = c->lat.dims[0] / 2;
      gg.dims[1] = c->lat.dims[1];
      gg.dims[2] = c->lat.dims[2];
      zb = zb || mrhs_zblock(gg, 16) > 0;
    }
    if (zb) cand.push_back({V_SMEM_ZB, 16});
    if (zb && prec != F64) cand.push_back({V_SMEM_PF_ZB, 16});
    if (tma_ok) {
      cand.push_back({V_TMA, 16});
      cand.push_back({V_TMA_TILE, 16});
    }
    if (pair_ok) {
      for (int ts : {8, 16, 32}) cand.push_back({V_PAIR, ts});
      if (zb) cand.push_back({V_PAIR_ZB, 16});
    }
  }
  if (tc_ok) cand.push_back({V_TC, tc_tile_sites()});
  const int plain_mode = mode & 31;  // without the fused reduction
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return dflt;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return dflt;
  }
  float best = 1e30f;
  TuneChoice pick = dflt;
  for (const TuneChoice& c : cand) {
    if (launch_variant(ctxs, prec, nrhs, a, dagger, plain_mode, c, c0->stream) != cudaSuccess) {
      cudaGetLastError();  // launch-configuration errors are not sticky: skip the candidate
      continue;
    }
    count_launch(c0, true);
    cudaEventRecord(e0, c0->stream);
    bool ok = true;
    for (int r = 0; r < 3 && ok; r++) {
      ok = launch_variant(ctxs, prec, nrhs, a, dagger, plain_mode, c, c0->stream) == cudaSuccess;
      count_launch(c0, true);
    }
    cudaEventRecord(e1, c0->stream);
    float ms = 0;
    if (!ok || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  tune_store(key, pick, best / 3);
  return pick;
}

wcl_status dslash_ex(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const FieldRef& out, const FieldRef& in,
                     const FieldRef* x, const FieldRef* out2, int out_parity, bool dagger, CloverSel post,
                     CloverSel pre, Coef alpha, Coef beta, const int* active, const EpiSpec* epi) {
  wcl_ctx* c0 = ctxs[0];
  const int dp = prec;
  DslashArgs a;
  memset(&a, 0, sizeof a);
  a.out = out;
  a.in = in;
  if (x) a.x = *x;
  if (out2) a.out2 = *out2;
  if (epi && epi->kind != EPI_NONE) {
    a.f = epi->f;
    a.partials = epi->partials;
    a.counters = epi->counters;
    a.sc = epi->sc;
    a.maxch = epi->maxch;
  }
  a.out_parity = out_parity;
  a.active = active;
  double sites = 0;
  for (size_t l = 0; l < ctxs.size(); l++) {
    const LatticeDevice& L = ctxs[l]->lat;
    a.gauge[l][0] = L.gauge[dp][0];
    a.gauge[l][1] = L.gauge[dp][1];
    const int p = out_parity;
    if (post) {
      a.cpost[l] = post == CL_A ? L.clov[dp][p] : L.clovinv[dp][p];
      a.cpost_norm[l] = post == CL_A ? L.clov_norm[dp * 2 + p] : L.clovinv_norm[dp * 2 + p];
    }
    if (pre) {
      a.cpre[l] = pre == CL_A ? L.clov[dp][p] : L.clovinv[dp][p];
      a.cpre_norm[l] = pre == CL_A ? L.clov_norm[dp * 2 + p] : L.clovinv_norm[dp * 2 + p];
    }
    a.alpha[l] = coef_value(alpha, L.kappa);
    a.beta[l] = coef_value(beta, L.kappa);
    sites += (double)L.vh * nrhs;
  }
  int mode = 0;
  if (post) mode |= MODE_POST;
  if (x) mode |= MODE_XPAY;
  if (x && pre) mode |= MODE_PRE;
  if (out2) mode |= MODE_RECON;
  const TuneChoice ch = choose_variant(ctxs, prec, nrhs, a, dagger, mode);
  if (epi) mode |= epi->kind << 5;
  wcl_ctx::Timed* t = prof_begin(c0);
  const cudaError_t e = launch_variant(ctxs, prec, nrhs, a, dagger, mode, ch, c0->stream);
  if (e != cudaSuccess) return cuda_fail(e, "dslash launch");
  count_launch(c0, true);
  if (ch.variant != V_THREAD && epi && epi->kind != EPI_NONE) count_launch(c0);  // finaliser
  if (t) {
    cudaEventRecord(t->b, c0->stream);
    double sp, lk, cl;
    spinor_site_bytes(prec, sp, lk, cl);
    double per = 8 * lk + 2 * sp + (post ? cl : 0) + (x ? sp : 0) + (x && pre ? cl : 0) + (out2 ? sp : 0) +
                 ((epi && epi->kind == EPI_ALPHA) ? sp : 0);
    // links and clover are shared by the right-hand sides of a site
    double per_site_shared = 8 * lk + (post ? cl : 0) + (x && pre ? cl : 0);
    double per_rhs = per - per_site_shared;
    double base_sites = sites / nrhs;
    t->bytes = base_sites * per_site_shared + sites * per_rhs;
    t->prec = prec;
    t->flops = sites * (1320.0 + (post ? 504.0 : 0.0) + ((x && pre) ? 504.0 : 0.0) + (x ? 48.0 : 0.0));
  }
  return WCL_OK;
}

wcl_status clover_apply(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const FieldRef& out,
                        const FieldRef& x, int parity, CloverSel which, const int* active) {
  wcl_ctx* c0 = ctxs[0];
  const int block = 128;
  CloverArgs a;
  memset(&a, 0, sizeof a);
  a.b = make_batch(ctxs, nrhs, block, 0);
  a.out = out;
  a.x = x;
  a.active = active;
  const int dp = prec;
  for (size_t l = 0; l < ctxs.size(); l++) {
    const LatticeDevice& L = ctxs[l]->lat;
    a.c[l] = which == CL_A ? L.clov[dp][parity] : L.clovinv[dp][parity];
    a.c_norm[l] = which == CL_A ? L.clov_norm[dp * 2 + parity] : L.clovinv_norm[dp * 2 + parity];
  }
  cudaError_t e;
  switch (prec) {
    case F64: e = launch_clover<F64>(a, block, c0->stream); break;
    case DF64: e = launch_clover<DF64>(a, block, c0->stream); break;
    case F32: e = launch_clover<F32>(a, block, c0->stream); break;
    case F16: e = launch_clover<F16>(a, block, c0->stream); break;
    default: e = launch_clover<BF16>(a, block, c0->stream); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "clover launch");
  count_launch(c0);
  return WCL_OK;
}

wcl_status apply_mhat(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const FieldRef& out_e,
                      const FieldRef& in_e, const FieldRef& tmp_o, bool dagger, const int* active,
                      const EpiSpec* epi) {
  // tmp_o = A_oo^-1 D_oe in_e
  WCL_CHECK(dslash(ctxs, prec, nrhs, tmp_o, in_e, nullptr, 1, dagger, CL_AINV, CL_NONE, C_ONE, C_ZERO, active));
  // out_e = A_ee in_e - kappa^2 D_eo tmp_o (+ the fused reduction)
  WCL_CHECK(dslash_ex(ctxs, prec, nrhs, out_e, tmp_o, &in_e, nullptr, 0, dagger, CL_NONE, CL_A, C_MKAPPA2, C_ONE,
                      active, epi));
  return WCL_OK;
}

template <int PO, int PI>
static cudaError_t run_convert(const Batch& b, const FieldRef& out, const FieldRef& in, const int* active, int block,
                               cudaStream_t st) {
  Convert<PO, PI> f;
  f.out = out;
  f.in = in;
  return run_map(b, f, active, block, st);
}

wcl_status convert(const std::vector<wcl_ctx*>& ctxs, int pout, int pin, int nrhs, const FieldRef& out,
                   const FieldRef& in, const int* active) {
  wcl_ctx* c0 = ctxs[0];
  const int block = c0->blas_block;
  Batch b = make_batch(ctxs, nrhs, block, RED_MAXCH);
  cudaError_t e = cudaErrorInvalidValue;
  const int key = (pout == DF64 || pin == DF64) ? 100 + pout * 8 + pin : pout * 4 + pin;
  switch (key) {
    case F32 * 4 + F64: e = run_convert<F32, F64>(b, out, in, active, block, c0->stream); break;
    case F16 * 4 + F64: e = run_convert<F16, F64>(b, out, in, active, block, c0->stream); break;
    case BF16 * 4 + F64: e = run_convert<BF16, F64>(b, out, in, active, block, c0->stream); break;
    case F64 * 4 + F32: e = run_convert<F64, F32>(b, out, in, active, block, c0->stream); break;
    case F64 * 4 + F16: e = run_convert<F64, F16>(b, out, in, active, block, c0->stream); break;
    case F64 * 4 + BF16: e = run_convert<F64, BF16>(b, out, in, active, block, c0->stream); break;
    case F64 * 4 + F64: e = run_convert<F64, F64>(b, out, in, active, block, c0->stream); break;
    case 100 + DF64 * 8 + F64: e = run_convert<DF64, F64>(b, out, in, active, block, c0->stream); break;
    case 100 + F64 * 8 + DF64: e = run_convert<F64, DF64>(b, out, in, active, block, c0->stream); break;
    case F32 * 4 + F32: e = run_convert<F32, F32>(b, out, in, active, block, c0->stream); break;
    case F16 * 4 + F16: e = run_convert<F16, F16>(b, out, in, active, block, c0->stream); break;
    case BF16 * 4 + BF16: e = run_convert<BF16, BF16>(b, out, in, active, block, c0->stream); break;
    default: set_error("conversion %d -> %d not instantiated", pin, pout); return WCL_ERR_INVALID_ARG;
  }
  if (e != cudaSuccess) return cuda_fail(e, "convert launch");
  count_launch(c0);
  return WCL_OK;
}

static void accum(wcl_ctx* c, size_t from, size_t to) {
  for (size_t k = from; k < to; k++) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[k].a, c->ev_pool[k].b) == cudaSuccess) {
      c->dslash_ms += ms;
      c->dslash_timed++;
      c->dslash_bytes += c->ev_pool[k].bytes;
      c->dslash_flops += c->ev_pool[k].flops;
      const int pr = c->ev_pool[k].prec;
      if (pr >= 0 && pr < 5) {
        c->prec_ms[pr] += ms;
        c->prec_timed[pr]++;
        c->prec_bytes[pr] += c->ev_pool[k].bytes;
        c->prec_flops[pr] += c->ev_pool[k].flops;
      }
    } else {
      cudaGetLastError();
    }
  }
}

void profile_flush(wcl_ctx* c, size_t from) {
  if (c->ev_used > from) accum(c, from, c->ev_used);
  c->ev_used = from;
}

wcl_status hws_get(wcl_ctx* c, const std::string& name, size_t bytes, void** out) {
  auto& b = c->hws[name];
  if (b.bytes < bytes) {
    if (b.p) {
      WCL_CUDA(cudaStreamSynchronize(c->stream));
      WCL_CUDA(cudaFreeHost(b.p));
      b.p = nullptr;
      b.bytes = 0;
    }
    WCL_CUDA(cudaMallocHost(&b.p, bytes));
    memset(b.p, 0, bytes);
    b.bytes = bytes;
  }
  *out = b.p;
  return WCL_OK;
}

void profile_accum_range(wcl_ctx* c, size_t from, size_t to) { accum(c, from, to); }

}  // namespace wcl
