// Library context: device data of one lattice, named workspace buffers, the
// internal work stream, profiling events and launch counters; plus the helpers
// that build batch geometry and launch the fused operator kernels.
#pragma once
#include <map>
#include <string>
#include <vector>

#include "../../include/wcl.h"
#include "blas.cuh"
#include "dslash.cuh"
#include "fields.cuh"

struct wcl_ctx {
  int device = 0;
  cudaStream_t user_stream = nullptr;  // caller's stream (may be the legacy default)
  cudaStream_t stream = nullptr;       // internal non-blocking stream all work runs on
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  wcl::LatticeDevice lat;
  struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
  };
  std::map<std::string, Buf> ws;   // workspace, grown on demand, freed in wcl_destroy
  std::map<std::string, Buf> hws;  // pinned host staging
  int* d_flags = nullptr;
  int* h_flags = nullptr;  // pinned

  // counters and profiling
  long long kernel_launches = 0, dslash_launches = 0, dslash_timed = 0;
  double dslash_ms = 0, dslash_bytes = 0, dslash_flops = 0;
  double prec_ms[5] = {}, prec_bytes[5] = {}, prec_flops[5] = {};
  long long prec_timed[5] = {};
  bool profiling = false;
  struct Timed {
    cudaEvent_t a, b;
    double bytes, flops;
    int prec;
  };
  std::vector<Timed> ev_pool;
  size_t ev_used = 0;
  bool capturing = false;
  long long capture_launches = 0, capture_dslash = 0;

  // learned preconditioner (PTC network) weights, device copies
  struct Ptc {
    float2* w32 = nullptr;          // FP32 complex master weights
    __nv_bfloat162* w16 = nullptr;  // BF16 copy used for inference
    float2* m = nullptr;            // Adam moments (re, im treated separately)
    float2* v = nullptr;
    double2* grad = nullptr;        // last gradient (dL/dRe + i dL/dIm)
    int steps = 0;
    bool loaded = false;
  } ptc;

  // launch shapes (picked by the tuner on first use)
  int dslash_block[4] = {128, 128, 128, 128};
  bool tensor_cores = false;  // multi-RHS 16-bit dslash on mma.sync (WCL_OPT_TENSOR_CORES)
  int shared_links = 16;      // multi-RHS dslash with links/clover staged in shared memory:
                              // 0 off, else its sites per CTA when the tuner does not choose
  bool autotune = true;       // time the dslash variants of a new configuration on first use
  int ptc_tensor_cores = 2;  // BF16 network layers' mixing: 0 SIMT, 1 mma.sync, 2 tcgen05
  int ptc_split = 1;         // BF16 terms per transported input on the tcgen05 layers
  bool wait_check = false;    // a kernel with bounded mbarrier waits ran since the last API return
  bool staged_spinors = false;   // untuned multi-RHS dslash: cp.async-staged neighbour spinors
  bool blocked_tiles = false;    // untuned multi-RHS dslash: tiles in z blocks (large lattices)
  bool paired_rhs = false;       // untuned multi-RHS FP32/16-bit dslash: the packed-pair kernel
  bool prefetch_spinors = false; // untuned multi-RHS dslash: next hop's spinor prefetched in registers
  int tma_staging = 0;           // untuned multi-RHS FP32 dslash: links and clover staged by TMA
                                 // (1 persistent CTAs, 2 one CTA per tile)
  int sloppy_updates = 0;        // 16-bit inner solves: updates above 10^-k ||b|| use the FP32 operator (0 off)
  int blas_block = 256;
  void* mg = nullptr;    // multigrid hierarchy (mg.cu), built by wcl_mg_setup
  void* stag = nullptr;  // staggered links and mass (stag.cu), loaded by wcl_load_staggered
};

namespace wcl {

void set_error(const char* fmt, ...);
wcl_status cuda_fail(cudaError_t e, const char* where);

#define WCL_CUDA(call)                                       \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail(_e, #call);      \
  } while (0)
#define WCL_CHECK(call)                  \
  do {                                   \
    wcl_status _s = (call);              \
    if (_s != WCL_OK) return _s;         \
  } while (0)

// named workspace buffer of at least `bytes`; zero-filled when (re)allocated
wcl_status ws_get(wcl_ctx* c, const std::string& name, size_t bytes, void** out);

// one field of precision prec with nrhs right-hand sides on every lattice of a batch
wcl_status ws_field(const std::vector<wcl_ctx*>& ctxs, const std::string& name, int prec, int nrhs, FieldRef* out);

// batch geometry for a launch with `block` threads; cap limits blocks per slice (grid-stride)
Batch make_batch(const std::vector<wcl_ctx*>& ctxs, int nrhs, int block, int cap);

// counts one launch (or, under graph capture, one captured node)
inline void count_launch(wcl_ctx* c, bool is_dslash = false) {
  if (c->capturing) {
    c->capture_launches++;
    c->capture_dslash += is_dslash;
  } else {
    c->kernel_launches++;
    c->dslash_launches += is_dslash;
  }
}

// coefficient selector for the per-lattice alpha / beta of the fused kernels
enum Coef { C_ZERO, C_ONE, C_KAPPA, C_MKAPPA, C_MKAPPA2 };
inline double coef_value(Coef c, double kappa) {
  switch (c) {
    case C_ZERO: return 0.0;
    case C_ONE: return 1.0;
    case C_KAPPA: return kappa;
    case C_MKAPPA: return -kappa;
    case C_MKAPPA2: return -kappa * kappa;
  }
  return 0.0;
}
enum CloverSel { CL_NONE = 0, CL_A = 1, CL_AINV = 2 };

// reduction fused into the epilogue of the second launch of M_hat (see DslashEpi)
struct EpiSpec {
  int kind = EPI_NONE;
  FieldRef f{};
  double* partials = nullptr;  // [slot][maxch][3]
  unsigned* counters = nullptr;
  Scalars* sc = nullptr;
  int maxch = 0;
};

// out_parity field = C_post(alpha D in + beta C_pre x) on all lattices of the batch
wcl_status dslash(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const FieldRef& out, const FieldRef& in,
                  const FieldRef* x, int out_parity, bool dagger, CloverSel post, CloverSel pre, Coef alpha,
                  Coef beta, const int* active);
// as dslash, with an optional second output: when out2 is given (post = A^-1,
// pre = A, x given) out = A^-1 t and out2 = t - A out for t = alpha D in + beta x
wcl_status dslash_ex(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const FieldRef& out, const FieldRef& in,
                     const FieldRef* x, const FieldRef* out2, int out_parity, bool dagger, CloverSel post,
                     CloverSel pre, Coef alpha, Coef beta, const int* active, const EpiSpec* epi = nullptr);
// blocks per (lattice, rhs) slice of a dslash launch (the epilogue partials need this many)
int dslash_max_chunks(const std::vector<wcl_ctx*>& ctxs, int prec);
// out = C x on parity `parity`
wcl_status clover_apply(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const FieldRef& out,
                        const FieldRef& x, int parity, CloverSel which, const int* active);
// M_hat (or its adjoint) in precision prec: out_e = A_ee in_e - kappa^2 D_eo A_oo^-1 D_oe in_e
wcl_status apply_mhat(const std::vector<wcl_ctx*>& ctxs, int prec, int nrhs, const FieldRef& out_e,
                      const FieldRef& in_e, const FieldRef& tmp_o, bool dagger, const int* active,
                      const EpiSpec* epi = nullptr);
// precision conversion of a parity field
wcl_status convert(const std::vector<wcl_ctx*>& ctxs, int pout, int pin, int nrhs, const FieldRef& out,
                   const FieldRef& in, const int* active);

// tensor-core multi-RHS dslash (dslash_tc.cu): 16-bit storage, 4 <= nrhs <= 16
cudaError_t launch_dslash_tc(int prec, const DslashArgs& a, bool dagger, int mode, cudaStream_t st);
int tc_tile_sites();
bool use_tc(const wcl_ctx* c, int prec, int nrhs, int mode);

// Autotuner: the dslash variant of a configuration (precision, mode, RHS count,
// lattice shapes, options) is picked by timing the candidates on first use and
// kept for the process; with WCL_TUNE_CACHE=<file> choices persist across runs.
// V_SMEM_ZB: the shared-memory kernel walking its tiles in z blocks (L2 reuse of the
// t neighbours on large lattices)
// V_PAIR / V_PAIR_ZB: the packed-pair kernel (dslash_pair.cuh: two right-hand sides per
// thread in float2 registers, FFMA2), in site order / z-blocked tile order
// V_SMEM_PF / V_SMEM_PF_ZB: the shared-memory kernel with the next hop's neighbour spinor
// loaded into registers while the current hop is computed
enum TuneVariant {
  V_THREAD = 0, V_SMEM = 1, V_TC = 2, V_SMEM_ASYNC = 3, V_SMEM_ZB = 4, V_PAIR = 5, V_PAIR_ZB = 6, V_SMEM_PF = 7,
  V_SMEM_PF_ZB = 8, V_TMA = 9, V_TMA_TILE = 10
};
// TMA-staged persistent multi-RHS kernel (dslash_tma.cu): FP32, one lattice with Lx = 32
bool tma_eligible(const LatGeom& g, int nrhs);
cudaError_t launch_dslash_tma(const DslashArgs& a, bool dagger, int mode, cudaStream_t st, int* err, bool persistent);
struct TuneChoice {
  int variant;  // TuneVariant
  int block;    // threads per CTA (V_THREAD) or sites per CTA (V_SMEM, V_SMEM_ASYNC, V_TC)
};
constexpr int kTuneMinBlock = 64;  // smallest per-thread block among the candidates
bool tune_lookup(const std::string& key, TuneChoice* out);
void tune_store(const std::string& key, TuneChoice c, float ms);
void tune_clear();  // forget every choice of this process (the file is left as it is)
bool use_mrhs(const wcl_ctx* c, int prec, int nrhs, int mode);

// per-precision instantiations (defined in dslash_<prec>.cu)
template <int P>
cudaError_t launch_dslash(const DslashArgs& a, bool dagger, int mode, int block, cudaStream_t st);
template <int P>
cudaError_t launch_clover(const CloverArgs& a, int block, cudaStream_t st);
// packed-pair multi-RHS kernel (FP32 and 16-bit storage; defined in dslash_<prec>.cu)
template <int P>
cudaError_t launch_dslash_pair(const DslashArgs& a, bool dagger, int mode, int ts, cudaStream_t st);
bool use_pair(const wcl_ctx* c, int prec, int nrhs, int mode);

// caller-owned QDP fields of a solve, one pointer per lattice
struct SolveIO {
  void* const* d_x;
  const void* const* d_b;
};

// accumulate the device times of profiled launches [from, used) and release them
// (call after a stream sync); profile_accum_range keeps them (graph-owned events)
void profile_flush(wcl_ctx* c, size_t from = 0);
void profile_accum_range(wcl_ctx* c, size_t from, size_t to);
// pinned host buffer, grown on demand
wcl_status hws_get(wcl_ctx* c, const std::string& name, size_t bytes, void** out);
// device address of wcl_apply_Mpc_noalloc's fixed scratch array, looked up once per
// device with that device current (loads its module, which allocates the array)
wcl_status noalloc_prepare(int device);
// load the module of the FP64 per-thread dslash kernels (dslash_f64.cu) without a launch
cudaError_t load_dslash_f64_module();
// multigrid (mg.cu): release the hierarchy; solve M x = b for right-hand side at complex
// offset rhs_off_c of the caller's QDP buffers by FGCR preconditioned with the K-cycle
void mg_free(wcl_ctx* c);
void stag_free(wcl_ctx* c);
// the batched K-cycle as a preconditioner of flexible GCR on M_hat (mg.cu): z_e = [K(r_e (+) 0)]_e
wcl_status mg_batched_cycle(wcl_ctx* c, int nrhs, const void* r_even, void* z_even);
wcl_status mg_solve_one(wcl_ctx* c, const void* d_b, void* d_x, long rhs_off_c, const wcl_solve_params& prm,
                        wcl_solve_info* info);

}  // namespace wcl
