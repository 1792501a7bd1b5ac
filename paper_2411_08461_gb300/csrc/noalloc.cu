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
// in `g_noalloc_scratch` below.
//
// The array belongs to this file's module.  Under CUDA's lazy module loading a
// module is loaded -- and its device arrays allocated -- the first time one of
// its symbols or kernels is touched, so the device address is looked up in
// wcl_create (noalloc_prepare below), where allocating is allowed, and the
// module of the FP64 operator kernels the call launches is loaded there too; the
// call itself only reads the cached address.  From then on the device holds the
// array until the process exits (or until a cudaDeviceReset, which invalidates
// it together with every other resource of the library's contexts).
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

// Set-up, once per device, with that device current (called by wcl_create):
// translate the array's host-side symbol into its device address.  This loads the
// module if it is not loaded yet, which allocates the array.
wcl_status noalloc_prepare(int device) {
  if (device < 0 || device >= 256) {
    set_error("wcl_create: device ordinal %d out of range of the no-allocation scratch table", device);
    return WCL_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    // the FP64 operator kernels the call launches live in another module: load it
    // here as well (the import and export kernels' module is loaded by wcl_load_gauge)
    e = load_dslash_f64_module();
    if (e != cudaSuccess) return cuda_fail(e, "loading the FP64 dslash module");
    g_noalloc_ptr[device] = p;
  }
  return WCL_OK;
}

static void* noalloc_scratch(int device) {
  if (device < 0 || device >= 256) return nullptr;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  return g_noalloc_ptr[device];
}

// device memory of the context's GPU (cudaPointerGetAttributes allocates nothing)
static bool device_buffer(const wcl_ctx* c, const void* p, const char* what) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    set_error("wcl_apply_Mpc_noalloc: %s is not a CUDA-accessible pointer", what);
    return false;
  }
  if ((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == c->device) return true;
  set_error("wcl_apply_Mpc_noalloc: %s is not device memory of the context's GPU", what);
  return false;
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
  if (!device_buffer(c, d_in_e, "d_in_e") || !device_buffer(c, d_out_e, "d_out_e")) return WCL_ERR_INVALID_ARG;
  void* base = noalloc_scratch(c->device);
  if (!base) {
    set_error("wcl_apply_Mpc_noalloc: the scratch array of device %d was not set up (wcl_create failed to)",
              c->device);
    return WCL_ERR_CUDA;
  }
  e = cudaEventRecord(c->ev_in, c->user_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_in, 0);
  if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
  set_error("");

  const long fb = 12L * 16 * c->lat.stride;  // bytes of one FP64 parity field at this lattice's stride
  FieldRef in{}, tmp{}, out{};
  in.ptr[0] = base;
  tmp.ptr[0] = static_cast<char*>(base) + fb;
  out.ptr[0] = static_cast<char*>(base) + 2 * fb;

  // No profiling events (creating one is a driver-side allocation) and no autotuning:
  // a configuration the tuner has not seen runs its default kernel instead of timing
  // candidates (which would create events, synchronise and may write the cache file).
  const bool prof = c->profiling, tune = c->autotune;
  c->profiling = false;
  c->autotune = false;
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
  c->autotune = tune;
  e = cudaEventRecord(c->ev_out, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->user_stream, c->ev_out, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess && s == WCL_OK) s = cuda_fail(e, "cudaStreamSynchronize");
  return s;
}
