// The C ABI of libwcl (declarations and documentation in include/wcl.h).
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include <vector>

#include "context.cuh"

namespace wcl {
const char* last_error_text();
template <int S>
wcl_status krylov_solve(const std::vector<wcl_ctx*>& ctxs, int nrhs, const wcl_solve_params& prm, const SolveIO& io,
                        wcl_solve_info* info);
}  // namespace wcl

using namespace wcl;

namespace wcl {
void ptc_free(wcl_ctx* c);
}

// order the call after the caller's pending work, run on the internal stream
wcl_status wcl_enter(wcl_ctx* c) {
  WCL_CUDA(cudaSetDevice(c->device));
  WCL_CUDA(cudaEventRecord(c->ev_in, c->user_stream));
  WCL_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  set_error("");
  return WCL_OK;
}

wcl_status wcl_leave(wcl_ctx* c, wcl_status s) {
  // later work on the caller's stream is ordered after this call's work
  cudaError_t e = cudaEventRecord(c->ev_out, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->user_stream, c->ev_out, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess && s == WCL_OK) return cuda_fail(e, "cudaStreamSynchronize");
  if (e == cudaSuccess && c->wait_check) {
    // bits 0x100 (TMA-staged dslash) and 0x200 (tcgen05 network layer): a CTA gave up
    // on an mbarrier wait and left its outputs unwritten
    c->wait_check = false;
    e = cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return s == WCL_OK ? cuda_fail(e, "reading the device error word") : s;
    const int f = c->h_flags[0];
    if (f & 0x300) {
      c->h_flags[0] = f & ~0x300;
      e = cudaMemcpyAsync(c->d_flags, c->h_flags, sizeof(int), cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (s == WCL_OK) {
        set_error("a bounded mbarrier wait expired in the %s; its outputs were not written",
                  (f & 0x200) ? "tcgen05 network layer" : "TMA-staged dslash");
        s = WCL_ERR_TIMEOUT;
      }
    }
  }
  return s;
}

namespace {

wcl_status enter(wcl_ctx* c) { return wcl_enter(c); }
wcl_status leave(wcl_ctx* c, wcl_status s) { return wcl_leave(c, s); }

bool valid_prec(int p) { return p >= WCL_F64 && p <= WCL_BF16; }
bool valid_apply_prec(int p) { return p >= WCL_F64 && p <= WCL_DF64; }

// A fermion buffer of the caller: device memory of the context's device, or
// page-locked host memory, which the import and export kernels read and write in
// place through its device alias (over the host link, no staging copy).
static bool field_ptr(const wcl_ctx* c, const void* p, const void** out, const char* what) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: not a CUDA-accessible pointer", what);
    return false;
  }
  if ((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == c->device) {
    *out = p;
    return true;
  }
  if (at.type == cudaMemoryTypeHost && at.devicePointer) {
    *out = at.devicePointer;
    return true;
  }
  set_error("%s: neither device memory of the context's GPU nor page-locked host memory", what);
  return false;
}
static bool field_ptr(const wcl_ctx* c, void* p, void** out, const char* what) {
  const void* q = nullptr;
  if (!field_ptr(c, static_cast<const void*>(p), &q, what)) return false;
  *out = const_cast<void*>(q);
  return true;
}

wcl_status alloc_lattice(wcl_ctx* c) {
  LatticeDevice& L = c->lat;
  for (int pr = 0; pr < 5; pr++)
    for (int p = 0; p < 2; p++) {
      WCL_CUDA(cudaMalloc(&L.gauge[pr][p], gauge_parity_bytes(pr, L.stride)));
      WCL_CUDA(cudaMalloc(&L.clov[pr][p], clover_parity_bytes(pr, L.stride)));
      WCL_CUDA(cudaMalloc(&L.clovinv[pr][p], clover_parity_bytes(pr, L.stride)));
      if (pr == F16 || pr == BF16) {
        WCL_CUDA(cudaMalloc(&L.clov_norm[pr * 2 + p], sizeof(float) * L.stride));
        WCL_CUDA(cudaMalloc(&L.clovinv_norm[pr * 2 + p], sizeof(float) * L.stride));
      }
    }
  return WCL_OK;
}

void free_lattice(wcl_ctx* c) {
  LatticeDevice& L = c->lat;
  for (int pr = 0; pr < 5; pr++)
    for (int p = 0; p < 2; p++) {
      cudaFree(L.gauge[pr][p]);
      cudaFree(L.clov[pr][p]);
      cudaFree(L.clovinv[pr][p]);
      L.gauge[pr][p] = L.clov[pr][p] = L.clovinv[pr][p] = nullptr;
    }
  for (int k = 0; k < 8; k++) {
    cudaFree(L.clov_norm[k]);
    cudaFree(L.clovinv_norm[k]);
    L.clov_norm[k] = L.clovinv_norm[k] = nullptr;
  }
  L.loaded = false;
}

}  // namespace

// fermion-style caller buffer (device or page-locked host) for the other translation units
bool wcl_resolve_field(const wcl_ctx* c, const void* p, const void** out, const char* what) {
  return field_ptr(c, p, out, what);
}

extern "C" {

void wcl_default_params(wcl_solve_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->solver = WCL_BICGSTAB;
  p->outer = WCL_DF64;
  p->sloppy = WCL_F32;
  p->tol = 1e-10;
  p->maxiter = 20000;
  p->delta_reliable = 0.1;
  p->restart_on_update = 0;
  p->gcr_nkrylov = 20;
  p->use_graphs = 1;
  p->check_every = 8;
}

const char* wcl_status_string(wcl_status s) {
  switch (s) {
    case WCL_OK: return "ok";
    case WCL_ERR_INVALID_ARG: return "invalid argument";
    case WCL_ERR_CUDA: return "CUDA error";
    case WCL_ERR_OOM: return "out of device memory";
    case WCL_ERR_NOT_CONVERGED: return "not converged";
    case WCL_ERR_BREAKDOWN: return "Krylov breakdown";
    case WCL_ERR_NONFINITE: return "non-finite value";
    case WCL_ERR_RECONSTRUCT: return "link not SU(3)";
    case WCL_ERR_TIMEOUT: return "device wait timed out";
    case WCL_ERR_NO_GAUGE: return "no gauge field loaded";
    case WCL_ERR_NO_PRECOND: return "no preconditioner weights loaded";
  }
  return "unknown status";
}

const char* wcl_last_error(void) { return last_error_text(); }

wcl_status wcl_create(wcl_ctx** out, const int dims[4], int t_boundary, int device, void* cuda_stream) {
  set_error("");
  if (!out || !dims) {
    set_error("wcl_create: null pointer");
    return WCL_ERR_INVALID_ARG;
  }
  *out = nullptr;
  long vol = 1;
  for (int d = 0; d < 4; d++) {
    if (dims[d] < 2) {
      set_error("wcl_create: extent %d of direction %d is below 2", dims[d], d);
      return WCL_ERR_INVALID_ARG;
    }
    vol *= dims[d];
  }
  if (dims[0] % 2) {
    set_error("wcl_create: Lx = %d must be even", dims[0]);
    return WCL_ERR_INVALID_ARG;
  }
  if (vol >= (1L << 31)) {
    set_error("wcl_create: volume too large");
    return WCL_ERR_INVALID_ARG;
  }
  if (t_boundary != 1 && t_boundary != -1) {
    set_error("wcl_create: t_boundary must be +1 or -1");
    return WCL_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    set_error("wcl_create: no CUDA device %d", device);
    return WCL_ERR_INVALID_ARG;
  }
  wcl_ctx* c = new (std::nothrow) wcl_ctx;
  if (!c) return WCL_ERR_OOM;
  c->device = device;
  c->user_stream = static_cast<cudaStream_t>(cuda_stream);
  for (int d = 0; d < 4; d++) c->lat.dims[d] = dims[d];
  c->lat.tb = t_boundary;
  c->lat.vh = vol / 2;
  c->lat.stride = (c->lat.vh + 63) / 64 * 64;
  wcl_status s = WCL_OK;
  do {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { s = cuda_fail(e, "cudaSetDevice"); break; }
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { s = cuda_fail(e, "cudaStreamCreate"); break; }
    e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
    if (e != cudaSuccess) { s = cuda_fail(e, "cudaEventCreate"); break; }
    e = cudaMalloc(&c->d_flags, 64);
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_flags, 64);
    if (e != cudaSuccess) { s = cuda_fail(e, "flag buffers"); break; }
    // the fixed scratch of wcl_apply_Mpc_noalloc is looked up (its module loaded) here,
    // where allocating is allowed, not inside that call
    s = noalloc_prepare(device);
  } while (0);
  if (s != WCL_OK) {
    wcl_destroy(c);
    return s;
  }
  *out = c;
  return WCL_OK;
}

// shared by the isotropic and anisotropic loaders: the operator is
// M = A - kappa H with the t hops of H weighted by tw and A built with csw_t on the
// planes that contain t and csw_s on the spatial planes
static wcl_status load_gauge(wcl_ctx* c, const void* d_gauge, double kappa, double tw, double csw_t, double csw_s,
                             const char* name) {
  WCL_CHECK(enter(c));
  if (!c->lat.gauge[0][0]) {
    wcl_status s = alloc_lattice(c);
    if (s != WCL_OK) {
      free_lattice(c);
      return s;
    }
  }
  c->lat.loaded = false;
  c->lat.kappa = kappa;
  c->lat.csw = csw_s;
  c->lat.csw_t = csw_t;
  c->lat.tw = tw;
  WCL_CUDA(cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  WCL_CUDA(import_gauge(c->lat, d_gauge, c->d_flags, c->stream));
  count_launch(c);
  WCL_CUDA(build_clover(c->lat, d_gauge, kappa, csw_t, csw_s, c->d_flags, c->stream));
  count_launch(c, false);
  WCL_CUDA(cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  WCL_CHECK(leave(c, WCL_OK));
  const int f = c->h_flags[0];
  if (f & 1) {
    set_error("%s: non-finite link entries", name);
    return WCL_ERR_NONFINITE;
  }
  if (f & 2) {
    set_error("%s: a link deviates from SU(3) by more than 1e-12", name);
    return WCL_ERR_RECONSTRUCT;
  }
  if (f & 4) {
    set_error("%s: singular clover block", name);
    return WCL_ERR_INVALID_ARG;
  }
  c->lat.loaded = true;
  return WCL_OK;
}

wcl_status wcl_load_gauge(wcl_ctx* c, const void* d_gauge, double kappa, double csw) {
  if (!c || !d_gauge) {
    set_error("wcl_load_gauge: null pointer");
    return WCL_ERR_INVALID_ARG;
  }
  if (!(kappa == kappa) || !(csw == csw)) {
    set_error("wcl_load_gauge: kappa or csw is NaN");
    return WCL_ERR_INVALID_ARG;
  }
  return load_gauge(c, d_gauge, kappa, 1.0, csw, csw, "wcl_load_gauge");
}

wcl_status wcl_load_gauge_aniso(wcl_ctx* c, const void* d_gauge, double kappa, double xi0, double nu, double csw_t,
                                double csw_r) {
  if (!c || !d_gauge) {
    set_error("wcl_load_gauge_aniso: null pointer");
    return WCL_ERR_INVALID_ARG;
  }
  if (!std::isfinite(kappa) || !std::isfinite(csw_t) || !std::isfinite(csw_r) || !std::isfinite(xi0) ||
      !std::isfinite(nu) || !(xi0 > 0) || !(nu > 0)) {
    set_error("wcl_load_gauge_aniso: kappa, c_sw^t, c_sw^r must be finite and xi0, nu positive");
    return WCL_ERR_INVALID_ARG;
  }
  // kappa [W_4 + (nu/xi0) sum_i W_i] = (kappa nu/xi0) [(xi0/nu) W_4 + sum_i W_i]; the clover
  // coefficients are rescaled by the same factor so that kappa' c' equals kappa c
  const double kl = kappa * nu / xi0, tw = xi0 / nu;
  return load_gauge(c, d_gauge, kl, tw, csw_t * tw, csw_r / nu, "wcl_load_gauge_aniso");
}

wcl_status wcl_apply_D(wcl_ctx* c, void* d_out, const void* d_in, wcl_prec prec, int nrhs) {
  if (!c || !d_out || !d_in || nrhs < 1 || nrhs > 64 || !valid_apply_prec(prec)) {
    set_error("wcl_apply_D: invalid argument");
    return WCL_ERR_INVALID_ARG;
  }
  if (!field_ptr(c, d_out, &d_out, "wcl_apply_D out") || !field_ptr(c, d_in, &d_in, "wcl_apply_D in"))
    return WCL_ERR_INVALID_ARG;
  if (!c->lat.loaded) {
    set_error("wcl_apply_D: no gauge field loaded");
    return WCL_ERR_NO_GAUGE;
  }
  WCL_CHECK(enter(c));
  std::vector<wcl_ctx*> v{c};
  const LatticeDevice& L = c->lat;
  FieldRef ie, io, oe, oo, pe, po, qe, qo;
  WCL_CHECK(ws_field(v, "D_in_e", F64, nrhs, &ie));
  WCL_CHECK(ws_field(v, "D_in_o", F64, nrhs, &io));
  WCL_CHECK(ws_field(v, "D_out_e", F64, nrhs, &oe));
  WCL_CHECK(ws_field(v, "D_out_o", F64, nrhs, &oo));
  const long rs = 2 * L.vh * 12;
  WCL_CUDA(import_fermion(L, d_in, rs, 0, nrhs, ie.ptr[0], nullptr, c->stream));
  WCL_CUDA(import_fermion(L, d_in, rs, L.vh * 12, nrhs, io.ptr[0], nullptr, c->stream));
  count_launch(c);
  count_launch(c);
  if (prec == WCL_F64) {
    pe = ie, po = io, qe = oe, qo = oo;
  } else {
    WCL_CHECK(ws_field(v, "D_pin_e", prec, nrhs, &pe));
    WCL_CHECK(ws_field(v, "D_pin_o", prec, nrhs, &po));
    WCL_CHECK(ws_field(v, "D_pout_e", prec, nrhs, &qe));
    WCL_CHECK(ws_field(v, "D_pout_o", prec, nrhs, &qo));
    WCL_CHECK(convert(v, prec, F64, nrhs, pe, ie, nullptr));
    WCL_CHECK(convert(v, prec, F64, nrhs, po, io, nullptr));
  }
  // out_p = A_pp in_p - kappa D_{p,1-p} in_{1-p}
  WCL_CHECK(dslash(v, prec, nrhs, qe, po, &pe, 0, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, nullptr));
  WCL_CHECK(dslash(v, prec, nrhs, qo, pe, &po, 1, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, nullptr));
  if (prec != WCL_F64) {
    WCL_CHECK(convert(v, F64, prec, nrhs, oe, qe, nullptr));
    WCL_CHECK(convert(v, F64, prec, nrhs, oo, qo, nullptr));
  }
  WCL_CUDA(export_fermion(L, oe.ptr[0], nrhs, d_out, rs, 0, c->stream));
  WCL_CUDA(export_fermion(L, oo.ptr[0], nrhs, d_out, rs, L.vh * 12, c->stream));
  count_launch(c);
  count_launch(c);
  wcl_status s = leave(c, WCL_OK);
  profile_flush(c, 0);
  return s;
}

wcl_status wcl_apply_Mpc(wcl_ctx* c, void* d_out_e, const void* d_in_e, wcl_prec prec, int nrhs, int dagger) {
  if (!c || !d_out_e || !d_in_e || nrhs < 1 || nrhs > 64 || !valid_apply_prec(prec)) {
    set_error("wcl_apply_Mpc: invalid argument");
    return WCL_ERR_INVALID_ARG;
  }
  if (!field_ptr(c, d_out_e, &d_out_e, "wcl_apply_Mpc out") || !field_ptr(c, d_in_e, &d_in_e, "wcl_apply_Mpc in"))
    return WCL_ERR_INVALID_ARG;
  if (!c->lat.loaded) {
    set_error("wcl_apply_Mpc: no gauge field loaded");
    return WCL_ERR_NO_GAUGE;
  }
  WCL_CHECK(enter(c));
  std::vector<wcl_ctx*> v{c};
  const LatticeDevice& L = c->lat;
  FieldRef ie, oe, pe, qe, tmp;
  const bool fp64_fields = prec == WCL_F64;
  WCL_CHECK(ws_field(v, "M_in", F64, nrhs, &ie));
  WCL_CHECK(ws_field(v, "M_out", F64, nrhs, &oe));
  WCL_CHECK(ws_field(v, "M_tmp", fp64_fields ? F64 : prec, nrhs, &tmp));
  const long rs = L.vh * 12;
  WCL_CUDA(import_fermion(L, d_in_e, rs, 0, nrhs, ie.ptr[0], nullptr, c->stream));
  count_launch(c);
  if (fp64_fields) {
    pe = ie, qe = oe;
  } else {
    WCL_CHECK(ws_field(v, "M_pin", prec, nrhs, &pe));
    WCL_CHECK(ws_field(v, "M_pout", prec, nrhs, &qe));
    WCL_CHECK(convert(v, prec, F64, nrhs, pe, ie, nullptr));
  }
  WCL_CHECK(apply_mhat(v, prec, nrhs, qe, pe, tmp, dagger != 0, nullptr));
  if (!fp64_fields) WCL_CHECK(convert(v, F64, prec, nrhs, oe, qe, nullptr));
  WCL_CUDA(export_fermion(L, oe.ptr[0], nrhs, d_out_e, rs, 0, c->stream));
  count_launch(c);
  wcl_status s = leave(c, WCL_OK);
  profile_flush(c, 0);
  return s;
}

static wcl_status propagator_call(wcl_ctx* c, void* dst, const void* src, int to_prop, const char* name) {
  if (!c || !dst || !src) {
    set_error("%s: invalid argument", name);
    return WCL_ERR_INVALID_ARG;
  }
  if (!field_ptr(c, dst, &dst, name) || !field_ptr(c, src, &src, name)) return WCL_ERR_INVALID_ARG;
  WCL_CHECK(enter(c));
  WCL_CUDA(propagator_layout(c->lat, src, dst, to_prop, c->stream));
  count_launch(c);
  return leave(c, WCL_OK);
}

wcl_status wcl_fermions_to_propagator(wcl_ctx* c, void* d_prop, const void* d_x12) {
  return propagator_call(c, d_prop, d_x12, 1, "wcl_fermions_to_propagator");
}

wcl_status wcl_propagator_to_fermions(wcl_ctx* c, void* d_x12, const void* d_prop) {
  return propagator_call(c, d_x12, d_prop, 0, "wcl_propagator_to_fermions");
}

static wcl_status check_params(const wcl_solve_params* p) {
  if (!p || (p->outer != WCL_F64 && p->outer != WCL_DF64) || !valid_prec(p->sloppy) || !(p->tol > 0) ||
      p->maxiter < 1 ||
      !(p->delta_reliable > 0 && p->delta_reliable < 1) || p->check_every < 1 || p->check_every > 1024) {
    set_error("invalid solve parameters (outer F64 or DF64, 0 < delta < 1, tol > 0)");
    return WCL_ERR_INVALID_ARG;
  }
  if (p->solver != WCL_BICGSTAB && p->solver != WCL_CGNR && p->solver != WCL_FGCR_LEARNED && p->solver != WCL_GCR &&
      p->solver != WCL_FGCR_MG && p->solver != WCL_FGCR_MG_BATCHED) {
    set_error("unknown solver %d", (int)p->solver);
    return WCL_ERR_INVALID_ARG;
  }
  return WCL_OK;
}

static wcl_status solve(const std::vector<wcl_ctx*>& v, int nrhs, const wcl_solve_params* p, void* const* d_x,
                        const void* const* d_b, wcl_solve_info* info) {
  if (p->solver == WCL_FGCR_LEARNED && !v[0]->ptc.loaded) {
    set_error("learned FGCR: no preconditioner weights loaded (wcl_precond_load / wcl_precond_train)");
    return WCL_ERR_NO_PRECOND;
  }
  if (p->solver == WCL_FGCR_MG_BATCHED) {
    if (p->sloppy != WCL_F32) {
      set_error("batched multigrid FGCR: sloppy precision must be WCL_F32");
      return WCL_ERR_INVALID_ARG;
    }
    if (!v[0]->mg) {
      set_error("batched multigrid FGCR: no multigrid hierarchy (wcl_mg_setup)");
      return WCL_ERR_NO_PRECOND;
    }
  }
  SolveIO io{d_x, d_b};
  switch (p->sloppy) {
    case WCL_F64: return krylov_solve<F64>(v, nrhs, *p, io, info);
    case WCL_F32: return krylov_solve<F32>(v, nrhs, *p, io, info);
    case WCL_F16: return krylov_solve<F16>(v, nrhs, *p, io, info);
    default: return krylov_solve<BF16>(v, nrhs, *p, io, info);
  }
}

wcl_status wcl_invert(wcl_ctx* c, void* d_x, const void* d_b, int nrhs, const wcl_solve_params* params,
                      wcl_solve_info* info) {
  if (!c || !d_x || !d_b || !info || nrhs < 1 || nrhs > 12) {
    set_error("wcl_invert: invalid argument (nrhs must be 1..12)");
    return WCL_ERR_INVALID_ARG;
  }
  WCL_CHECK(check_params(params));
  if (!c->lat.loaded) {
    set_error("wcl_invert: no gauge field loaded");
    return WCL_ERR_NO_GAUGE;
  }
  if (!field_ptr(c, d_x, &d_x, "wcl_invert x") || !field_ptr(c, d_b, &d_b, "wcl_invert b"))
    return WCL_ERR_INVALID_ARG;
  WCL_CHECK(enter(c));
  if (params->solver == WCL_FGCR_MG) {
    // one right-hand side after the other through the multigrid-preconditioned FGCR
    const auto t0 = std::chrono::steady_clock::now();
    wcl_status worst = WCL_OK;
    for (int k = 0; k < nrhs && worst != WCL_ERR_NO_PRECOND; k++) {
      wcl_status s = mg_solve_one(c, d_b, d_x, (long)k * 2 * c->lat.vh * 12, *params, &info[k]);
      if (s != WCL_OK) return leave(c, s);
      if (worst == WCL_OK && info[k].status != WCL_OK) worst = (wcl_status)info[k].status;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < nrhs; k++) info[k].seconds = secs;
    if (worst != WCL_OK) set_error("right-hand side did not reach the tolerance (multigrid FGCR)");
    return leave(c, worst);
  }
  std::vector<wcl_ctx*> v{c};
  void* xs[1] = {d_x};
  const void* bs[1] = {d_b};
  wcl_status s = solve(v, nrhs, params, xs, bs, info);
  return leave(c, s);
}

wcl_status wcl_invert_batch(wcl_ctx* const* ctxs, int nctx, void* const* d_x, const void* const* d_b, int nrhs,
                            const wcl_solve_params* params, wcl_solve_info* info) {
  if (!ctxs || !d_x || !d_b || !info || nctx < 1 || nctx > MAXLAT || nrhs < 1 || nrhs > 12) {
    set_error("wcl_invert_batch: invalid argument (1 <= nctx <= 8, 1 <= nrhs <= 12)");
    return WCL_ERR_INVALID_ARG;
  }
  WCL_CHECK(check_params(params));
  if (params->solver == WCL_FGCR_MG || params->solver == WCL_FGCR_MG_BATCHED) {
    set_error("wcl_invert_batch: the multigrid solvers run through wcl_invert, one lattice at a time");
    return WCL_ERR_INVALID_ARG;
  }
  std::vector<wcl_ctx*> v;
  for (int i = 0; i < nctx; i++) {
    if (!ctxs[i] || !d_x[i] || !d_b[i]) {
      set_error("wcl_invert_batch: null entry %d", i);
      return WCL_ERR_INVALID_ARG;
    }
    if (ctxs[i]->device != ctxs[0]->device) {
      set_error("wcl_invert_batch: contexts on different devices");
      return WCL_ERR_INVALID_ARG;
    }
    for (int j = 0; j < i; j++)
      if (ctxs[j] == ctxs[i]) {
        set_error("wcl_invert_batch: context %d repeated", i);
        return WCL_ERR_INVALID_ARG;
      }
    if (!ctxs[i]->lat.loaded) {
      set_error("wcl_invert_batch: no gauge field loaded on context %d", i);
      return WCL_ERR_NO_GAUGE;
    }
    v.push_back(ctxs[i]);
  }
  std::vector<void*> xs(nctx);
  std::vector<const void*> bs(nctx);
  for (int i = 0; i < nctx; i++)
    if (!field_ptr(ctxs[i], d_x[i], &xs[i], "wcl_invert_batch x") ||
        !field_ptr(ctxs[i], d_b[i], &bs[i], "wcl_invert_batch b"))
      return WCL_ERR_INVALID_ARG;
  for (int i = 0; i < nctx; i++) {
    WCL_CHECK(enter(ctxs[i]));
    if (i) {
      // everything runs on the first context's stream
      WCL_CUDA(cudaEventRecord(ctxs[i]->ev_in, ctxs[i]->user_stream));
      WCL_CUDA(cudaStreamWaitEvent(ctxs[0]->stream, ctxs[i]->ev_in, 0));
    }
  }
  wcl_status s = solve(v, nrhs, params, xs.data(), bs.data(), info);
  return leave(ctxs[0], s);
}

wcl_status wcl_set_option(wcl_ctx* c, int option, int value) {
  if (!c) return WCL_ERR_INVALID_ARG;
  switch (option) {
    case WCL_OPT_TENSOR_CORES: c->tensor_cores = value != 0; return WCL_OK;
    case WCL_OPT_SHARED_LINKS:
      if (value == 0 || value == 1 || value == 8 || value == 16 || value == 32) {
        c->shared_links = value == 1 ? 16 : value;
        return WCL_OK;
      }
      break;
    case WCL_OPT_AUTOTUNE: c->autotune = value != 0; return WCL_OK;
    case WCL_OPT_PTC_TENSOR_CORES:
      if (value < 0 || value > 2) break;
      c->ptc_tensor_cores = value;
      return WCL_OK;
    case WCL_OPT_STAGED_SPINORS: c->staged_spinors = value != 0; return WCL_OK;
    case WCL_OPT_BLOCKED_TILES: c->blocked_tiles = value != 0; return WCL_OK;
    case WCL_OPT_PAIRED_RHS: c->paired_rhs = value != 0; return WCL_OK;
    case WCL_OPT_PREFETCH_SPINORS: c->prefetch_spinors = value != 0; return WCL_OK;
    case WCL_OPT_TMA_STAGING:
      if (value >= 0 && value <= 2) {
        c->tma_staging = value;
        return WCL_OK;
      }
      break;
    case WCL_OPT_PTC_SPLIT:
      if (value >= 1 && value <= 3) {
        c->ptc_split = value;
        return WCL_OK;
      }
      break;
    case WCL_OPT_SLOPPY_UPDATES:
      if (value >= 0 && value <= 8) {
        c->sloppy_updates = value;
        return WCL_OK;
      }
      break;
  }
  set_error("wcl_set_option: unknown option %d or value %d", option, value);
  return WCL_ERR_INVALID_ARG;
}

wcl_status wcl_set_profiling(wcl_ctx* c, int enable) {
  if (!c) return WCL_ERR_INVALID_ARG;
  c->profiling = enable != 0;
  return WCL_OK;
}

wcl_status wcl_get_stats(wcl_ctx* c, wcl_stats* out, int reset) {
  if (!c || !out) return WCL_ERR_INVALID_ARG;
  out->kernel_launches = c->kernel_launches;
  out->dslash_launches = c->dslash_launches;
  out->dslash_ms = c->dslash_ms;
  out->dslash_timed = c->dslash_timed;
  out->dslash_bytes = c->dslash_bytes;
  out->dslash_flops = c->dslash_flops;
  for (int k = 0; k < 5; k++) {
    out->prec_ms[k] = c->prec_ms[k];
    out->prec_timed[k] = c->prec_timed[k];
    out->prec_bytes[k] = c->prec_bytes[k];
    out->prec_flops[k] = c->prec_flops[k];
  }
  if (reset) {
    c->kernel_launches = c->dslash_launches = c->dslash_timed = 0;
    c->dslash_ms = c->dslash_bytes = c->dslash_flops = 0;
    for (int k = 0; k < 5; k++) {
      c->prec_ms[k] = c->prec_bytes[k] = c->prec_flops[k] = 0;
      c->prec_timed[k] = 0;
    }
  }
  return WCL_OK;
}

wcl_status wcl_destroy(wcl_ctx* c) {
  if (!c) return WCL_OK;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_lattice(c);
  ptc_free(c);
  mg_free(c);
  stag_free(c);
  for (auto& kv : c->ws) cudaFree(kv.second.p);
  for (auto& kv : c->hws) cudaFreeHost(kv.second.p);
  for (auto& t : c->ev_pool) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  if (c->d_flags) cudaFree(c->d_flags);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->stream) cudaStreamDestroy(c->stream);
  cudaGetLastError();
  delete c;
  return WCL_OK;
}

}  // extern "C"
