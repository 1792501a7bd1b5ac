// Learned preconditioner: weights, network application, loss/gradient and
// Adam training, all on the device (see ptc.cuh for the layer).
//
// The network acts on fields of the even-odd system: an even-parity residual
// is embedded in a whole-lattice field (odd sites zero), passed through the four
// layers, and the even part of the output approximates M_hat^-1 r.  Training
// minimises L = (1/B) sum_b ||N(r_b)_e - e_b||^2 / ||e_b||^2 over (r, e) pairs.
#include <cmath>
#include <cstring>
#include <vector>

#include "ptc.cuh"

namespace wcl {

// ---------------------------------------------------------------------------
// small kernels

// QDP even half [n][vh][12] complex128 -> full layout [n][1][2][6][stride] float4 (odd = 0)
__global__ void ptc_import_even_kernel(const double2* __restrict__ src, long vh, long stride, int n,
                                       float4* __restrict__ dst) {
  const long tot = (long)n * vh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / vh);
    const long i = idx % vh;
    const double2* s = src + ((size_t)r * vh + i) * 12;
    float4* de = dst + ptc_field_offset(r, 0, 1, 0, stride);
    float4* dodd = dst + ptc_field_offset(r, 0, 1, 1, stride);
    for (int k = 0; k < 6; k++) {
      double2 a = s[2 * k], b = s[2 * k + 1];
      de[k * stride + i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
      dodd[k * stride + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// full layout channel 0, even parity -> QDP even half complex128
__global__ void ptc_export_even_kernel(const float4* __restrict__ src, long vh, long stride, int n,
                                       double2* __restrict__ dst) {
  const long tot = (long)n * vh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / vh);
    const long i = idx % vh;
    const float4* s = src + ptc_field_offset(r, 0, 1, 0, stride);
    double2* d = dst + ((size_t)r * vh + i) * 12;
    for (int k = 0; k < 6; k++) {
      float4 v = s[k * stride + i];
      d[2 * k] = make_double2(v.x, v.y);
      d[2 * k + 1] = make_double2(v.z, v.w);
    }
  }
}

// parity field (SpinorIO<F32> layout [rhs][6][stride]) -> full layout even part, odd zero; and back
__global__ void ptc_embed_kernel(const float4* __restrict__ src, long vh, long stride, int n, float4* __restrict__ dst) {
  const long tot = (long)n * vh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / vh);
    const long i = idx % vh;
    const float4* s = src + (size_t)r * 6 * stride;
    float4* de = dst + ptc_field_offset(r, 0, 1, 0, stride);
    float4* dodd = dst + ptc_field_offset(r, 0, 1, 1, stride);
    for (int k = 0; k < 6; k++) {
      de[k * stride + i] = s[k * stride + i];
      dodd[k * stride + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}
__global__ void ptc_extract_kernel(const float4* __restrict__ src, long vh, long stride, int n, float4* __restrict__ dst) {
  const long tot = (long)n * vh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / vh);
    const long i = idx % vh;
    const float4* s = src + ptc_field_offset(r, 0, 1, 0, stride);
    float4* d = dst + (size_t)r * 6 * stride;
    for (int k = 0; k < 6; k++) d[k * stride + i] = s[k * stride + i];
  }
}

// ||e_b||^2 over the even sites (atomic FP64 sum per pair; a monitor value)
__global__ void ptc_norm_kernel(const float4* __restrict__ e, long vh, long stride, int n, double* __restrict__ out) {
  const long tot = (long)n * vh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / vh);
    const long i = idx % vh;
    const float4* s = e + ptc_field_offset(r, 0, 1, 0, stride);
    double acc = 0;
    for (int k = 0; k < 6; k++) {
      float4 v = s[k * stride + i];
      acc += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
    }
    atomicAdd(out + r, acc);
  }
}

// G = 2 (y - e) / (B ||e||^2) on even sites (0 on odd), loss += ||y - e||^2 / (B ||e||^2)
__global__ void ptc_loss_kernel(const float4* __restrict__ y, const float4* __restrict__ e, const double* __restrict__ en,
                                long vh, long stride, int n, float4* __restrict__ g, double* __restrict__ loss) {
  const long tot = (long)n * vh;
  double acc = 0;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < tot; idx += (long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / vh);
    const long i = idx % vh;
    const float4* ys = y + ptc_field_offset(r, 0, 1, 0, stride);
    const float4* es = e + ptc_field_offset(r, 0, 1, 0, stride);
    float4* ge = g + ptc_field_offset(r, 0, 1, 0, stride);
    float4* go = g + ptc_field_offset(r, 0, 1, 1, stride);
    const double sc = 1.0 / ((double)n * en[r]);
    double part = 0;
    for (int k = 0; k < 6; k++) {
      float4 a = ys[k * stride + i], b = es[k * stride + i];
      float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
      part += (double)d.x * d.x + (double)d.y * d.y + (double)d.z * d.z + (double)d.w * d.w;
      const float f = (float)(2.0 * sc);
      ge[k * stride + i] = make_float4(f * d.x, f * d.y, f * d.z, f * d.w);
      go[k * stride + i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    acc += part * sc;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// W'[ci][co][sbar] = W[co][ci][s]^+  (input gradient of a layer as another layer)
__global__ void ptc_adjoint_kernel(const float2* __restrict__ w, int cin, int cout, float2* __restrict__ wt) {
  const int tot = cout * cin * PTC_NSHIFT * 16;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
    int e = idx;
    const int b = e % 4; e /= 4;
    const int a = e % 4; e /= 4;
    const int s = e % PTC_NSHIFT; e /= PTC_NSHIFT;
    const int ci = e % cin;
    const int co = e / cin;
    const int sbar = (s == 0) ? 0 : (((s - 1) & 1) ? s - 1 : s + 1);
    const float2 v = w[idx];
    // destination layer has cin' = cout, cout' = cin: index ((ci * cout + co) * 9 + sbar) * 16 + b * 4 + a
    wt[((ci * cout + co) * PTC_NSHIFT + sbar) * 16 + b * 4 + a] = make_float2(v.x, -v.y);
  }
}

// sum weight-gradient partials over (parity, slot, chunk): grad[co][ci][s][a][b]
__global__ void ptc_grad_sum_kernel(const double2* __restrict__ parts, int nslot, int cin, int cout, int maxch,
                                    int nchunk, size_t parity_stride, double2* __restrict__ grad) {
  const int tot = cout * cin * PTC_NSHIFT * 16;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
    const int ab = idx % 16;
    const int s = (idx / 16) % PTC_NSHIFT;
    const int ci = (idx / (16 * PTC_NSHIFT)) % cin;
    const int co = idx / (16 * PTC_NSHIFT * cin);
    const int cs = ci * PTC_NSHIFT + s;
    double re = 0, im = 0;
    for (int p = 0; p < 2; p++)
      for (int sl = 0; sl < nslot; sl++)
        for (int c = 0; c < nchunk; c++) {
          const double2 v = parts[p * parity_stride + (((size_t)sl * (cin * PTC_NSHIFT) + cs) * maxch + c) * (cout * 16) +
                                  co * 16 + ab];
          re += v.x;
          im += v.y;
        }
    grad[idx] = make_double2(re, im);
  }
}

// Adam on real and imaginary parts; refresh the BF16 copy
__global__ void ptc_adam_kernel(float2* __restrict__ w, float2* __restrict__ m, float2* __restrict__ v,
                                const double2* __restrict__ g, int n, float lr, float b1, float b2, float eps,
                                float c1, float c2, __nv_bfloat162* __restrict__ wb) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const float gr = (float)g[k].x, gi = (float)g[k].y;
    float2 mm = m[k], vv = v[k], ww = w[k];
    mm.x = b1 * mm.x + (1 - b1) * gr;
    mm.y = b1 * mm.y + (1 - b1) * gi;
    vv.x = b2 * vv.x + (1 - b2) * gr * gr;
    vv.y = b2 * vv.y + (1 - b2) * gi * gi;
    ww.x -= lr * (mm.x / c1) / (sqrtf(vv.x / c2) + eps);
    ww.y -= lr * (mm.y / c1) / (sqrtf(vv.y / c2) + eps);
    m[k] = mm;
    v[k] = vv;
    w[k] = ww;
    wb[k] = __floats2bfloat162_rn(ww.x, ww.y);
  }
}

__global__ void ptc_to_bf16_kernel(const float2* __restrict__ w, int n, __nv_bfloat162* __restrict__ wb) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    wb[k] = __floats2bfloat162_rn(w[k].x, w[k].y);
}

static int grid_for(long n, int block) {
  long g = (n + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------------------
// host helpers

wcl_status ptc_alloc(wcl_ctx* c) {
  auto& P = c->ptc;
  if (P.w32) return WCL_OK;
  const int n = ptc_total_weights();
  WCL_CUDA(cudaMalloc(&P.w32, sizeof(float2) * n));
  WCL_CUDA(cudaMalloc(&P.w16, sizeof(__nv_bfloat162) * n));
  WCL_CUDA(cudaMalloc(&P.m, sizeof(float2) * n));
  WCL_CUDA(cudaMalloc(&P.v, sizeof(float2) * n));
  WCL_CUDA(cudaMalloc(&P.grad, sizeof(double2) * n));
  WCL_CUDA(cudaMemsetAsync(P.m, 0, sizeof(float2) * n, c->stream));
  WCL_CUDA(cudaMemsetAsync(P.v, 0, sizeof(float2) * n, c->stream));
  return WCL_OK;
}

void ptc_free(wcl_ctx* c) {
  auto& P = c->ptc;
  cudaFree(P.w32);
  cudaFree(P.w16);
  cudaFree(P.m);
  cudaFree(P.v);
  cudaFree(P.grad);
  P = wcl_ctx::Ptc{};
}

// one layer on both parities (or only `only_parity` >= 0)
static wcl_status layer_both(const std::vector<wcl_ctx*>& ctxs, int nrhs, const float4* const* in, float4* const* out,
                             int cin, int cout, const float2* w, const __nv_bfloat162* wb, int use_bf16,
                             int only_parity = -1) {
  wcl_ctx* c0 = ctxs[0];
  PtcLayerArgs a;
  memset(&a, 0, sizeof a);
  a.b = make_batch(ctxs, nrhs, ptc_layer_sites_per_cta(), 0);
  for (size_t l = 0; l < ctxs.size(); l++) {
    a.in[l] = in[l];
    a.out[l] = out[l];
    a.gauge[l][0] = ctxs[l]->lat.gauge[F32][0];
    a.gauge[l][1] = ctxs[l]->lat.gauge[F32][1];
  }
  a.w = w;
  a.wb = wb;
  a.cin = cin;
  a.cout = cout;
  a.use_bf16 = use_bf16;
  if (use_bf16 && c0->ptc_tensor_cores == 2) {
    // tcgen05 layers: 128-site tiles, B operands of the nine shifts packed once per layer
    a.b = make_batch(ctxs, nrhs, ptc_umma_sites_per_cta(), 0);
    void* q;
    WCL_CHECK(ws_get(c0, "ptc_umma_b", ptc_umma_pack_bytes(PTC_MAXC, PTC_MAXC), &q));
    uint4* bp = static_cast<uint4*>(q);
    cudaError_t e = ptc_pack_umma(wb, cin, cout, bp, c0->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ptc tcgen05 operand packing");
    count_launch(c0);
    c0->wait_check = true;
    for (int p = 0; p < 2; p++) {
      if (only_parity >= 0 && p != only_parity) continue;
      a.parity = p;
      e = ptc_layer_umma(a, bp, c0->ptc_split, c0->d_flags, c0->stream);
      if (e != cudaSuccess) return cuda_fail(e, "ptc tcgen05 layer launch");
      count_launch(c0);
    }
    return WCL_OK;
  }
  uint4* frag = nullptr;
  if (use_bf16 && c0->ptc_tensor_cores == 1) {
    void* q;
    WCL_CHECK(ws_get(c0, "ptc_frag", sizeof(uint4) * ptc_frag_entries(PTC_MAXC, PTC_MAXC), &q));
    frag = static_cast<uint4*>(q);
    cudaError_t e = ptc_pack_frag(wb, cin, cout, frag, c0->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ptc fragment packing");
    count_launch(c0);
  }
  for (int p = 0; p < 2; p++) {
    if (only_parity >= 0 && p != only_parity) continue;
    a.parity = p;
    cudaError_t e = ptc_layer(a, c0->stream, frag);
    if (e != cudaSuccess) return cuda_fail(e, "ptc layer launch");
    count_launch(c0);
  }
  return WCL_OK;
}

// N(r) for parity fields r (F32, [rhs][6][stride]) on every lattice of the batch -> z (same layout)
wcl_status ptc_apply(const std::vector<wcl_ctx*>& ctxs, int nrhs, const FieldRef& r, const FieldRef& z, int use_bf16) {
  wcl_ctx* c0 = ctxs[0];
  if (!c0->ptc.loaded) {
    set_error("learned preconditioner: no weights loaded (wcl_precond_load or wcl_precond_train)");
    return WCL_ERR_NO_PRECOND;
  }
  const float4 *in[MAXLAT], *xa[MAXLAT], *ya[MAXLAT];
  float4 *inw[MAXLAT], *xw[MAXLAT], *yw[MAXLAT], *ow[MAXLAT];
  for (size_t l = 0; l < ctxs.size(); l++) {
    wcl_ctx* c = ctxs[l];
    const long st = c->lat.stride;
    void *p1, *p2, *p3, *p4;
    const size_t one = (size_t)nrhs * 2 * 6 * st * sizeof(float4);
    WCL_CHECK(ws_get(c, "ptc_in", one, &p1));
    WCL_CHECK(ws_get(c, "ptc_x", one * PTC_MAXC, &p2));
    WCL_CHECK(ws_get(c, "ptc_y", one * PTC_MAXC, &p3));
    WCL_CHECK(ws_get(c, "ptc_out", one, &p4));
    inw[l] = static_cast<float4*>(p1);
    in[l] = inw[l];
    xw[l] = static_cast<float4*>(p2);
    xa[l] = xw[l];
    yw[l] = static_cast<float4*>(p3);
    ya[l] = yw[l];
    ow[l] = static_cast<float4*>(p4);
    ptc_embed_kernel<<<grid_for((long)nrhs * c->lat.vh, 256), 256, 0, c0->stream>>>(
        static_cast<const float4*>(r.ptr[l]), c->lat.vh, st, nrhs, inw[l]);
    WCL_CUDA(cudaGetLastError());
    count_launch(c0);
  }
  const auto& P = c0->ptc;
  WCL_CHECK(layer_both(ctxs, nrhs, in, xw, 1, 4, P.w32 + ptc_layer_offset(0), P.w16 + ptc_layer_offset(0), use_bf16));
  WCL_CHECK(layer_both(ctxs, nrhs, xa, yw, 4, 4, P.w32 + ptc_layer_offset(1), P.w16 + ptc_layer_offset(1), use_bf16));
  WCL_CHECK(layer_both(ctxs, nrhs, ya, xw, 4, 4, P.w32 + ptc_layer_offset(2), P.w16 + ptc_layer_offset(2), use_bf16));
  WCL_CHECK(layer_both(ctxs, nrhs, xa, ow, 4, 1, P.w32 + ptc_layer_offset(3), P.w16 + ptc_layer_offset(3), use_bf16,
                       /*only even output*/ 0));
  for (size_t l = 0; l < ctxs.size(); l++) {
    wcl_ctx* c = ctxs[l];
    ptc_extract_kernel<<<grid_for((long)nrhs * c->lat.vh, 256), 256, 0, c0->stream>>>(
        ow[l], c->lat.vh, c->lat.stride, nrhs, static_cast<float4*>(z.ptr[l]));
    WCL_CUDA(cudaGetLastError());
    count_launch(c0);
  }
  return WCL_OK;
}

// Loss and gradient over `n` pairs held as full-layout fields R, E (single lattice ctx).
// Activations of the forward pass are kept for the backward pass.  Gradient left in c->ptc.grad.
static wcl_status ptc_loss_grad_dev(wcl_ctx* c, const float4* R, const float4* E, int n, double* h_loss) {
  std::vector<wcl_ctx*> v{c};
  const long st = c->lat.stride, vh = c->lat.vh;
  const size_t one = (size_t)n * 2 * 6 * st * sizeof(float4);
  void* q;
  float4* acts[PTC_NLAYER + 1];
  float4* grads[PTC_NLAYER + 1];
  acts[0] = const_cast<float4*>(R);
  for (int l = 1; l <= PTC_NLAYER; l++) {
    WCL_CHECK(ws_get(c, "ptc_act" + std::to_string(l), one * PTC_CH[l], &q));
    acts[l] = static_cast<float4*>(q);
    WCL_CHECK(ws_get(c, "ptc_g" + std::to_string(l), one * PTC_CH[l], &q));
    grads[l] = static_cast<float4*>(q);
  }
  WCL_CHECK(ws_get(c, "ptc_wadj", sizeof(float2) * PTC_MAXC * PTC_MAXC * PTC_NSHIFT * 16, &q));
  float2* wadj = static_cast<float2*>(q);
  WCL_CHECK(ws_get(c, "ptc_scal", sizeof(double) * (n + 1), &q));
  double* en = static_cast<double*>(q);
  double* dloss = en + n;
  const int gblock = 128, maxch = 64;
  Batch gb = make_batch(v, n, gblock, maxch);
  const size_t pstride = (size_t)n * (PTC_MAXC * PTC_NSHIFT) * maxch * (PTC_MAXC * 16);
  WCL_CHECK(ws_get(c, "ptc_parts", sizeof(double2) * 2 * pstride, &q));
  double2* parts = static_cast<double2*>(q);
  auto& P = c->ptc;

  // forward (FP32 master weights)
  for (int l = 0; l < PTC_NLAYER; l++) {
    const float4* in[1] = {acts[l]};
    float4* out[1] = {acts[l + 1]};
    WCL_CHECK(layer_both(v, n, in, out, PTC_CH[l], PTC_CH[l + 1], P.w32 + ptc_layer_offset(l),
                         P.w16 + ptc_layer_offset(l), 0));
  }
  // loss and output gradient
  WCL_CUDA(cudaMemsetAsync(en, 0, sizeof(double) * (n + 1), c->stream));
  ptc_norm_kernel<<<grid_for((long)n * vh, 256), 256, 0, c->stream>>>(E, vh, st, n, en);
  ptc_loss_kernel<<<grid_for((long)n * vh, 256), 256, 0, c->stream>>>(acts[PTC_NLAYER], E, en, vh, st, n,
                                                                     grads[PTC_NLAYER], dloss);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  count_launch(c);
  // backward
  for (int l = PTC_NLAYER - 1; l >= 0; l--) {
    const int cin = PTC_CH[l], cout = PTC_CH[l + 1];
    PtcGradArgs ga;
    memset(&ga, 0, sizeof ga);
    ga.b = gb;
    ga.in[0] = acts[l];
    ga.g[0] = grads[l + 1];
    ga.gauge[0][0] = c->lat.gauge[F32][0];
    ga.gauge[0][1] = c->lat.gauge[F32][1];
    ga.cin = cin;
    ga.cout = cout;
    ga.maxch = maxch;
    for (int p = 0; p < 2; p++) {
      ga.parity = p;
      ga.partials = parts + p * pstride;
      WCL_CUDA(ptc_grad(ga, gblock, c->stream));
      count_launch(c);
    }
    const int nw = cout * cin * PTC_NSHIFT * 16;
    int maxnch = 0;
    for (int k = 0; k < gb.nlat; k++) maxnch = std::max(maxnch, gb.lat[k].nchunk);
    ptc_grad_sum_kernel<<<grid_for(nw, 128), 128, 0, c->stream>>>(parts, n, cin, cout, maxch, maxnch, pstride,
                                                                  P.grad + ptc_layer_offset(l));
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    if (l > 0) {
      ptc_adjoint_kernel<<<grid_for(nw, 128), 128, 0, c->stream>>>(P.w32 + ptc_layer_offset(l), cin, cout, wadj);
      WCL_CUDA(cudaGetLastError());
      count_launch(c);
      const float4* in[1] = {grads[l + 1]};
      float4* out[1] = {grads[l]};
      WCL_CHECK(layer_both(v, n, in, out, cout, cin, wadj, nullptr, 0));
    }
  }
  if (h_loss) {
    WCL_CUDA(cudaMemcpyAsync(h_loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  return WCL_OK;
}

static wcl_status import_pairs(wcl_ctx* c, const void* d_r, const void* d_e, int n, const float4** R, const float4** E) {
  const long st = c->lat.stride, vh = c->lat.vh;
  const size_t one = (size_t)n * 2 * 6 * st * sizeof(float4);
  void *pr, *pe;
  WCL_CHECK(ws_get(c, "ptc_pairs_r", one, &pr));
  WCL_CHECK(ws_get(c, "ptc_pairs_e", one, &pe));
  ptc_import_even_kernel<<<grid_for((long)n * vh, 256), 256, 0, c->stream>>>(static_cast<const double2*>(d_r), vh,
                                                                             st, n, static_cast<float4*>(pr));
  ptc_import_even_kernel<<<grid_for((long)n * vh, 256), 256, 0, c->stream>>>(static_cast<const double2*>(d_e), vh,
                                                                             st, n, static_cast<float4*>(pe));
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  count_launch(c);
  *R = static_cast<const float4*>(pr);
  *E = static_cast<const float4*>(pe);
  return WCL_OK;
}

}  // namespace wcl

using namespace wcl;

wcl_status wcl_enter(wcl_ctx* c);
wcl_status wcl_leave(wcl_ctx* c, wcl_status s);

extern "C" {

wcl_status wcl_precond_load(wcl_ctx* c, const double* h_weights) {
  if (!c || !h_weights) {
    set_error("wcl_precond_load: null pointer");
    return WCL_ERR_INVALID_ARG;
  }
  WCL_CHECK(wcl_enter(c));
  WCL_CHECK(ptc_alloc(c));
  const int n = ptc_total_weights();
  std::vector<float2> w(n);
  for (int k = 0; k < n; k++) {
    const double re = h_weights[2 * k], im = h_weights[2 * k + 1];
    if (!std::isfinite(re) || !std::isfinite(im)) {
      set_error("wcl_precond_load: non-finite weight %d", k);
      return WCL_ERR_NONFINITE;
    }
    w[k] = make_float2((float)re, (float)im);
  }
  WCL_CUDA(cudaMemcpyAsync(c->ptc.w32, w.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, c->stream));
  ptc_to_bf16_kernel<<<grid_for(n, 256), 256, 0, c->stream>>>(c->ptc.w32, n, c->ptc.w16);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  WCL_CUDA(cudaMemsetAsync(c->ptc.m, 0, sizeof(float2) * n, c->stream));
  WCL_CUDA(cudaMemsetAsync(c->ptc.v, 0, sizeof(float2) * n, c->stream));
  c->ptc.steps = 0;
  c->ptc.loaded = true;
  return wcl_leave(c, WCL_OK);
}

wcl_status wcl_precond_get(wcl_ctx* c, double* h_weights) {
  if (!c || !h_weights) return WCL_ERR_INVALID_ARG;
  if (!c->ptc.loaded) {
    set_error("wcl_precond_get: no weights");
    return WCL_ERR_NO_PRECOND;
  }
  WCL_CHECK(wcl_enter(c));
  const int n = ptc_total_weights();
  std::vector<float2> w(n);
  WCL_CUDA(cudaMemcpyAsync(w.data(), c->ptc.w32, sizeof(float2) * n, cudaMemcpyDeviceToHost, c->stream));
  WCL_CHECK(wcl_leave(c, WCL_OK));
  for (int k = 0; k < n; k++) {
    h_weights[2 * k] = w[k].x;
    h_weights[2 * k + 1] = w[k].y;
  }
  return WCL_OK;
}

wcl_status wcl_precond_apply(wcl_ctx* c, void* d_out_e, const void* d_in_e, int nrhs, int bf16) {
  if (!c || !d_out_e || !d_in_e || nrhs < 1 || nrhs > 64) {
    set_error("wcl_precond_apply: invalid argument");
    return WCL_ERR_INVALID_ARG;
  }
  if (!c->lat.loaded) {
    set_error("wcl_precond_apply: no gauge field loaded");
    return WCL_ERR_NO_GAUGE;
  }
  WCL_CHECK(wcl_enter(c));
  std::vector<wcl_ctx*> v{c};
  FieldRef in64, in32, out32;
  WCL_CHECK(ws_field(v, "P_in64", F64, nrhs, &in64));
  WCL_CHECK(ws_field(v, "P_in32", F32, nrhs, &in32));
  WCL_CHECK(ws_field(v, "P_out32", F32, nrhs, &out32));
  const long rs = c->lat.vh * 12;
  WCL_CUDA(import_fermion(c->lat, d_in_e, rs, 0, nrhs, in64.ptr[0], nullptr, c->stream));
  count_launch(c);
  WCL_CHECK(convert(v, F32, F64, nrhs, in32, in64, nullptr));
  WCL_CHECK(ptc_apply(v, nrhs, in32, out32, bf16));
  WCL_CHECK(convert(v, F64, F32, nrhs, in64, out32, nullptr));
  WCL_CUDA(export_fermion(c->lat, in64.ptr[0], nrhs, d_out_e, rs, 0, c->stream));
  count_launch(c);
  return wcl_leave(c, WCL_OK);
}

wcl_status wcl_precond_loss_grad(wcl_ctx* c, const void* d_r_e, const void* d_e_e, int npairs, double* loss,
                                 double* h_grad) {
  if (!c || !d_r_e || !d_e_e || npairs < 1 || !loss) {
    set_error("wcl_precond_loss_grad: invalid argument");
    return WCL_ERR_INVALID_ARG;
  }
  if (!c->lat.loaded) return WCL_ERR_NO_GAUGE;
  if (!c->ptc.loaded) {
    set_error("wcl_precond_loss_grad: no weights loaded");
    return WCL_ERR_NO_PRECOND;
  }
  WCL_CHECK(wcl_enter(c));
  const float4 *R, *E;
  WCL_CHECK(import_pairs(c, d_r_e, d_e_e, npairs, &R, &E));
  WCL_CHECK(ptc_loss_grad_dev(c, R, E, npairs, loss));
  const int n = ptc_total_weights();
  std::vector<double2> g(n);
  if (h_grad) WCL_CUDA(cudaMemcpyAsync(g.data(), c->ptc.grad, sizeof(double2) * n, cudaMemcpyDeviceToHost, c->stream));
  WCL_CHECK(wcl_leave(c, WCL_OK));
  if (h_grad)
    for (int k = 0; k < n; k++) {
      h_grad[2 * k] = g[k].x;
      h_grad[2 * k + 1] = g[k].y;
    }
  return WCL_OK;
}

wcl_status wcl_precond_train(wcl_ctx* c, const void* d_r_e, const void* d_e_e, int npairs,
                             const wcl_train_params* tp, double* h_loss_per_epoch) {
  if (!c || !d_r_e || !d_e_e || !tp || npairs < 1 || tp->epochs < 1 || tp->batch < 1 || !(tp->lr > 0)) {
    set_error("wcl_precond_train: invalid argument");
    return WCL_ERR_INVALID_ARG;
  }
  if (!c->lat.loaded) return WCL_ERR_NO_GAUGE;
  if (!c->ptc.loaded) {
    set_error("wcl_precond_train: load initial weights first (wcl_precond_load)");
    return WCL_ERR_NO_PRECOND;
  }
  WCL_CHECK(wcl_enter(c));
  const float4 *R, *E;
  WCL_CHECK(import_pairs(c, d_r_e, d_e_e, npairs, &R, &E));
  const long st = c->lat.stride;
  const size_t pair_f4 = (size_t)2 * 6 * st;
  const int nw = ptc_total_weights();
  for (int ep = 0; ep < tp->epochs; ep++) {
    double ep_loss = 0;
    int nb = 0;
    for (int b0 = 0; b0 < npairs; b0 += tp->batch) {
      const int n = std::min(tp->batch, npairs - b0);
      double bl = 0;
      WCL_CHECK(ptc_loss_grad_dev(c, R + b0 * pair_f4, E + b0 * pair_f4, n, &bl));
      auto& P = c->ptc;
      P.steps++;
      const float c1 = 1.f - powf((float)tp->beta1, (float)P.steps), c2 = 1.f - powf((float)tp->beta2, (float)P.steps);
      ptc_adam_kernel<<<grid_for(nw, 256), 256, 0, c->stream>>>(P.w32, P.m, P.v, P.grad, nw, (float)tp->lr,
                                                                (float)tp->beta1, (float)tp->beta2, (float)tp->eps,
                                                                c1, c2, P.w16);
      WCL_CUDA(cudaGetLastError());
      count_launch(c);
      WCL_CUDA(cudaStreamSynchronize(c->stream));
      ep_loss += bl;
      nb++;
    }
    if (h_loss_per_epoch) h_loss_per_epoch[ep] = ep_loss / nb;
  }
  return wcl_leave(c, WCL_OK);
}

void wcl_default_train_params(wcl_train_params* p) {
  if (!p) return;
  p->epochs = 4;
  p->batch = 8;
  p->lr = 1e-3;
  p->beta1 = 0.9;
  p->beta2 = 0.999;
  p->eps = 1e-8;
}

}  // extern "C"
