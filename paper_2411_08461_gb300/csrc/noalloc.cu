// wcl_apply_Mpc_noalloc: the FP64 Schur operator with all of its scratch in a
// fixed, file-scope device array instead of library workspace.
//
// Why it exists: some host programs cannot let a library call cudaMalloc at
// call time -- for example a program that hands all device memory to its own
// pool allocator up front, or a latency-sensitive loop that cannot afford the
// device synchronisation and possible failure of an allocation in the middle
// of a run.  This entry point allocates nothing: the caller passes the input
// and output, the gauge field and clover term come from wcl_load_gauge (done
// earlier, outside the constrained region), and the intermediate fields live
// in `g_noalloc_scratch` below, which every GPU that loads this library holds
// until the process exits.
//
// The scratch holds three FP64 parity fields (input copy, odd-parity
// intermediate A_oo^-1 D_oe x, output) of at most WCL_NOALLOC_MAX_VH sites.
// Each call writes every element it later reads, so nothing needs clearing,
// but the contents of the previous call remain in the array.  All calls share
// the one array: calls whose GPU work overlaps (different streams, threads or
// contexts on the same device) race on it and must be serialised by the caller.
#include <mutex>

#include "context.cuh"

namespace wcl {

constexpr long NOALLOC_FIELD_BYTES = 12L * 16 * WCL_NOALLOC_MAX_VH;  // one FP64 parity field
constexpr long NOALLOC_BYTES = 3 * NOALLOC_FIELD_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};  // device address of the scratch array, per device ordinal
}  // namespace

// One-time set-up per device (the device must be current): translate the
// array's host-side symbol into its device address.
static wcl_status noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= 256) {
    set_error("wcl_apply_Mpc_noalloc: device ordinal %d out of range", device);
    return WCL_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return WCL_OK;
}

}  // namespace wcl

using namespace wcl;

extern "C" wcl_status wcl_apply_Mpc_noalloc(wcl_ctx* c, void* d_out_e, const void* d_in_e, int dagger) {
  if (!c || !d_out_e || !d_in_e) {
    set_error("wcl_apply_Mpc_noalloc: null pointer");
    return WCL_ERR_INVALID_ARG;
  }
  if (!c->lat.loaded) {
    set_error("wcl_apply_Mpc_noalloc: no gauge field loaded");
    return WCL_ERR_NO_GAUGE;
  }
  if (c->lat.stride > WCL_NOALLOC_MAX_VH) {
    set_error("wcl_apply_Mpc_noalloc: %ld sites per parity (padded %ld) exceed the fixed scratch of %d sites",
              (long)c->lat.vh, (long)c->lat.stride, (int)WCL_NOALLOC_MAX_VH);
    return WCL_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  void* base = nullptr;
  WCL_CHECK(noalloc_scratch(c->device, &base));
  e = cudaEventRecord(c->ev_in, c->user_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_in, 0);
  if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
  set_error("");

  const long fb = 12L * 16 * c->lat.stride;  // bytes of one FP64 parity field at this lattice's stride
  FieldRef in{}, tmp{}, out{};
  in.ptr[0] = base;
  tmp.ptr[0] = static_cast<char*>(base) + fb;
  out.ptr[0] = static_cast<char*>(base) + 2 * fb;

  const bool prof = c->profiling;
  c->profiling = false;  // event creation would be a driver-side allocation
  std::vector<wcl_ctx*> v{c};
  const long rs = c->lat.vh * 12;
  wcl_status s = WCL_OK;
  e = import_fermion(c->lat, d_in_e, rs, 0, 1, in.ptr[0], nullptr, c->stream);
  if (e != cudaSuccess) s = cuda_fail(e, "import");
  if (s == WCL_OK) {
    count_launch(c);
    s = apply_mhat(v, F64, 1, out, in, tmp, dagger != 0, nullptr);
  }
  if (s == WCL_OK) {
    e = export_fermion(c->lat, out.ptr[0], 1, d_out_e, rs, 0, c->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "export");
    else count_launch(c);
  }
  c->profiling = prof;
  e = cudaEventRecord(c->ev_out, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->user_stream, c->ev_out, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess && s == WCL_OK) s = cuda_fail(e, "cudaStreamSynchronize");
  return s;
}
