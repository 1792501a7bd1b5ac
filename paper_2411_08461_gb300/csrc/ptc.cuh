// Gauge-covariant parallel-transport (PTC) network: the learned preconditioner
// of flexible GCR.  The paper has no learned component; the layer is
//
//   out_{c'}(x) = sum_{c, s} W[c', c, s] (T_s in_c)(x),   s in {0, +x, -x, ..., +t, -t}
//   T_0 psi(x) = psi(x),  T_+mu psi(x) = eta U_mu(x) psi(x+mu),
//   T_-mu psi(x) = eta U_mu(x-mu)^+ psi(x-mu),
//
// W[c', c, s] a complex 4x4 spin matrix, eta the fermion time-boundary sign.
// Channels 1 -> 4 -> 4 -> 4 -> 1, no nonlinearity.  Because T_s^+ = T_{-s}, the
// input gradient of a layer is the same layer with W'[c, c', -s] = W[c', c, s]^+,
// so one kernel serves forward and backward.
//
// Device layout of a multi-channel full-lattice field (FP32):
//   [rhs][channel][parity][6 float4 chunks][stride]   (chunk layout of SpinorIO<F32>)
#pragma once
#include "context.cuh"

namespace wcl {

constexpr int PTC_NLAYER = 4;
constexpr int PTC_NSHIFT = 9;
constexpr int PTC_CH[PTC_NLAYER + 1] = {1, 4, 4, 4, 1};
constexpr int PTC_MAXC = 4;

// complex weights of one layer as 4x4 blocks: index ((co * cin + ci) * 9 + s) * 16 + a * 4 + b
inline int ptc_layer_offset(int layer) {
  int off = 0;
  for (int l = 0; l < layer; l++) off += PTC_CH[l] * PTC_CH[l + 1] * PTC_NSHIFT * 16;
  return off;
}
inline int ptc_total_weights() { return ptc_layer_offset(PTC_NLAYER); }

struct PtcLayerArgs {
  Batch b;               // slices = (lattice, rhs); out parity given below
  const float4* in[MAXLAT];   // [rhs][cin][parity][6][stride]
  float4* out[MAXLAT];        // [rhs][cout][parity][6][stride]
  const void* gauge[MAXLAT][2];
  const float2* w;       // FP32 complex weights of this layer (master copy)
  const __nv_bfloat162* wb;  // BF16 copy (used when use_bf16)
  int cin, cout;
  int parity;            // output parity
  int use_bf16;
  int accumulate;        // out += instead of out =
};

// channel-c, parity-p chunk base of a multi-channel field for one rhs
__host__ __device__ inline size_t ptc_field_offset(int rhs, int c, int nch, int parity, long stride) {
  return ((size_t)(rhs * nch + c) * 2 + parity) * 6 * (size_t)stride;
}

// a.b must be built with ptc_layer_sites_per_cta() sites per block.  With frag
// (the layer's packed A fragments, ptc_pack_frag) and a.use_bf16 the mixing runs on
// the tensor cores; otherwise the FP32 SIMT layer.
cudaError_t ptc_layer(const PtcLayerArgs& a, cudaStream_t st, const uint4* frag = nullptr);
int ptc_layer_sites_per_cta();
// BF16 weights of one layer -> A fragments of the tensor-core layer (ptc_frag_entries uint4)
int ptc_frag_entries(int cin, int cout);
cudaError_t ptc_pack_frag(const __nv_bfloat162* wb, int cin, int cout, uint4* frag, cudaStream_t st);

// tcgen05 layer: a.b built with ptc_umma_sites_per_cta() sites per block; bpack the
// layer's B operands (ptc_pack_umma, ptc_umma_pack_bytes bytes); nparts = 1, 2 or 3 BF16
// terms per transported input; a wait that expires sets bit 0x200 of *err
int ptc_umma_sites_per_cta();
size_t ptc_umma_pack_bytes(int cin, int cout);
cudaError_t ptc_pack_umma(const __nv_bfloat162* wb, int cin, int cout, uint4* out, cudaStream_t st);
cudaError_t ptc_layer_umma(const PtcLayerArgs& a, const uint4* bpack, int nparts, int* err, cudaStream_t st);

// dW[co][ci][s] += sum_x G_co(x) (T_s in_ci)(x)^+  (colour summed), per slice;
// writes per-block partials [slot][ci*9+s][chunk][co][16] as float2 (FP32)
struct PtcGradArgs {
  Batch b;
  const float4* in[MAXLAT];
  const float4* g[MAXLAT];
  const void* gauge[MAXLAT][2];
  int cin, cout, parity;
  double2* partials;  // [slot][cin*9][maxch][cout*16]
  int maxch;
};
cudaError_t ptc_grad(const PtcGradArgs& a, int block, cudaStream_t st);

}  // namespace wcl
