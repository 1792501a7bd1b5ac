// Device-resident lattice data of one context and the one-time set-up kernels.
#pragma once
#include "internal.cuh"

namespace wcl {

struct LatticeDevice {
  int dims[4] = {0, 0, 0, 0};
  int tb = -1;          // fermion time boundary (+1 / -1)
  long vh = 0;          // sites per parity
  long stride = 0;      // padded sites per chunk
  double kappa = 0, csw = 0;
  double csw_t = 0;     // clover coefficient of the planes that contain t (csw: the spatial planes)
  double tw = 1.0;      // t-hop weight: xi_0 / nu of the anisotropic operator (kappa holds kappa nu / xi_0)
  bool loaded = false;
  // [prec][parity], prec = F64, F32, F16, BF16, DF64 (the FP64 values split into float pairs)
  void* gauge[5][2] = {};    // links, [mu][chunk][stride]; 18 reals (FP64, DF64) or 12 (row 2 rebuilt)
  void* clov[5][2] = {};     // A (packed Hermitian blocks)
  void* clovinv[5][2] = {};  // A^-1
  float* clov_norm[8] = {};  // [prec*2 + parity], half precisions only
  float* clovinv_norm[8] = {};
};

// bytes of one parity-field chunk array for precision P (without norms)
inline size_t spinor_field_bytes(int prec, long stride) {
  switch (prec) {
    case F64:
    case DF64: return (size_t)12 * 16 * stride;
    case F32: return (size_t)6 * 16 * stride;
    default: return (size_t)3 * 16 * stride;
  }
}
inline size_t gauge_parity_bytes(int prec, long stride) {
  switch (prec) {
    case F64:
    case DF64: return (size_t)4 * 9 * 16 * stride;
    case F32: return (size_t)4 * 3 * 16 * stride;
    default: return (size_t)4 * 3 * 8 * stride;
  }
}
inline size_t clover_parity_bytes(int prec, long stride) {
  switch (prec) {
    case F64:
    case DF64: return (size_t)36 * 16 * stride;
    case F32: return (size_t)18 * 16 * stride;
    default: return (size_t)9 * 16 * stride;
  }
}

// 12 fermion fields (sources k = 3 spin + colour) <-> one propagator field, QDP layouts
cudaError_t propagator_layout(const LatticeDevice& L, const void* src, void* dst, int to_prop, cudaStream_t st);

// d_flags bits: 1 non-finite input, 2 link not SU(3), 4 singular clover block
cudaError_t import_gauge(const LatticeDevice& L, const void* d_qdp, int* d_flags, cudaStream_t st);
cudaError_t build_clover(const LatticeDevice& L, const void* d_qdp, double kappa, double csw_t, double csw_s,
                         int* d_flags,
                         cudaStream_t st);
// complex-element strides: rhs_stride_c between right-hand sides, par_off_c to the parity block
cudaError_t import_fermion(const LatticeDevice& L, const void* d_src, long rhs_stride_c, long par_off_c, int nrhs,
                           void* d_dst64, int* d_flags, cudaStream_t st);
cudaError_t export_fermion(const LatticeDevice& L, const void* d_src64, int nrhs, void* d_dst, long rhs_stride_c,
                           long par_off_c, cudaStream_t st);

}  // namespace wcl
