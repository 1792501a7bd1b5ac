// Staggered operator of the HISQ action on given smeared links, and its solve.
//
//   M chi = 2 m chi + D chi
//   D chi(x) = sum_mu eta_mu(x) [ V_mu(x) chi(x + mu) - V_mu(x - mu)^+ chi(x - mu)
//                               + W_mu(x) chi(x + 3 mu) - W_mu(x - 3 mu)^+ chi(x - 3 mu) ]
//
// V are the fat (one-hop) links and W the long (three-hop, Naik coefficient included)
// links the HISQ smearing produces; eta are the MILC staggered phases (Sec. II.A:
// eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z)), and every hop
// across t = Lt - 1 -> 0 carries the fermion time boundary sign.  CG is the paper's
// default solver for HISQ (Sec. II.E).  D maps one parity to the other (1 and 3 are
// odd), so with mass m > 0 the solve runs on the even sites:
//   (4 m^2 - D_eo D_oe) x_e = 2 m b_e - D_eo b_o,     x_o = (b_o - D_oe x_e) / (2 m),
// a Hermitian positive definite system (D is anti-Hermitian), by CG in FP32 between
// IEEE FP64 restarts from the true residual ||b - M x|| of the whole system.
//
// Layouts: caller fields are QDP [2][Lt][Lz][Ly][Lx/2][3] complex128; links are the QDP
// gauge layout [4][2][Lt][Lz][Ly][Lx/2][3][3] complex128 (not SU(3): all 18 reals kept).
// Internally, per parity: vectors [3 colour][stride] (double2 or float2), links
// [mu][9 entries][stride]; one thread per (output site, right-hand side).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "context.cuh"

wcl_status wcl_enter(wcl_ctx* c);
wcl_status wcl_leave(wcl_ctx* c, wcl_status s);
bool wcl_resolve_field(const wcl_ctx* c, const void* p, const void** out, const char* what);

namespace wcl {

struct StagGeom {
  int dims[4];
  int lxh;
  long vh, stride;
  float tb_f;
  double tb;
};

struct StagState {
  StagGeom g{};
  double mass = 0;
  void* V[2][2] = {};  // [prec F64 = 0, F32 = 1][parity]
  void* W[2][2] = {};
  double* part = nullptr;
  std::vector<double> hpart;
  bool loaded = false;
};
constexpr int STAG_PART = 1024;

template <typename R>
struct V2;
template <>
struct V2<double> {
  using T = double2;
};
template <>
struct V2<float> {
  using T = float2;
};

__device__ __forceinline__ void stag_coords(const StagGeom& g, int p, long i, int c[4]) {
  const int xh = (int)(i % g.lxh);
  long rem = i / g.lxh;
  c[1] = (int)(rem % g.dims[1]);
  rem /= g.dims[1];
  c[2] = (int)(rem % g.dims[2]);
  c[3] = (int)(rem / g.dims[2]);
  c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
}
__device__ __forceinline__ long stag_cb(const StagGeom& g, const int c[4]) {
  return (((long)c[3] * g.dims[2] + c[2]) * g.dims[1] + c[1]) * g.lxh + c[0] / 2;
}

// links: QDP gauge (complex128) -> [mu][9][stride] per parity, FP64 and FP32
__global__ void stag_links_kernel(const double2* __restrict__ q, StagGeom g, double2* __restrict__ d0,
                                  double2* __restrict__ d1, float2* __restrict__ f0, float2* __restrict__ f1,
                                  int* __restrict__ flags) {
  const long n = 4 * 2 * g.vh * 9;
  bool fin = true;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int k = (int)(e % 9);
    long rest = e / 9;
    const long i = rest % g.vh;
    rest /= g.vh;
    const int p = (int)(rest % 2);
    const int mu = (int)(rest / 2);
    const double2 v = q[(((long)mu * 2 + p) * g.vh + i) * 9 + k];
    fin = fin && isfinite(v.x) && isfinite(v.y);
    const long o = ((long)mu * 9 + k) * g.stride + i;
    (p ? d1 : d0)[o] = v;
    (p ? f1 : f0)[o] = make_float2((float)v.x, (float)v.y);
  }
  if (!fin) atomicOr(flags, 1);
}

// vectors: QDP (complex128, [2][vh][3]) <-> internal full FP64 [2][3][stride]
__global__ void stag_import_kernel(const double2* __restrict__ q, StagGeom g, double2* __restrict__ d,
                                   int* __restrict__ flags) {
  const long n = 2 * g.vh * 3;
  bool fin = true;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int a = (int)(e % 3);
    const long site = e / 3;
    const int p = (int)(site / g.vh);
    const long i = site % g.vh;
    const double2 v = q[e];
    fin = fin && isfinite(v.x) && isfinite(v.y);
    d[((long)p * 3 + a) * g.stride + i] = v;
  }
  if (!fin && flags) atomicOr(flags, 1);
}
__global__ void stag_export_kernel(const double2* __restrict__ d, StagGeom g, double2* __restrict__ q) {
  const long n = 2 * g.vh * 3;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int a = (int)(e % 3);
    const long site = e / 3;
    const int p = (int)(site / g.vh);
    const long i = site % g.vh;
    q[e] = d[((long)p * 3 + a) * g.stride + i];
  }
}

template <typename T>
__device__ __forceinline__ T cm(T a, T b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename T>
__device__ __forceinline__ T cmc(T a, T b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }  // conj(a) b

// out = alpha D in + beta x on the sites of parity p (in: parity 1 - p; x: parity p or null)
template <typename R>
__global__ void __launch_bounds__(128) stag_dslash_kernel(const __grid_constant__ StagGeom g, int p,
                                                          const typename V2<R>::T* __restrict__ V0,
                                                          const typename V2<R>::T* __restrict__ V1,
                                                          const typename V2<R>::T* __restrict__ W0,
                                                          const typename V2<R>::T* __restrict__ W1,
                                                          const typename V2<R>::T* __restrict__ in,
                                                          const typename V2<R>::T* __restrict__ x,
                                                          typename V2<R>::T* __restrict__ out, R alpha, R beta,
                                                          int nrhs, long rhs_stride) {
  using T = typename V2<R>::T;
  const long total = (long)nrhs * g.vh;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int r = (int)(e / g.vh);
    const long i = e % g.vh;
    const T* inr = in + r * rhs_stride;
    int c[4];
    stag_coords(g, p, i, c);
    const T* Vh = p ? V1 : V0;  // links at this site
    const T* Vt = p ? V0 : V1;  // links at the neighbours (other parity)
    const T* Wh = p ? W1 : W0;
    const T* Wt = p ? W0 : W1;
    T acc[3] = {{0, 0}, {0, 0}, {0, 0}};
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      R eta = 1;
      if (mu == 1) eta = (c[0] & 1) ? -1 : 1;
      if (mu == 2) eta = ((c[0] + c[1]) & 1) ? -1 : 1;
      if (mu == 3) eta = ((c[0] + c[1] + c[2]) & 1) ? -1 : 1;
      const int L = g.dims[mu];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int n = h ? 3 : 1;
        const T* Lh = h ? Wh : Vh;
        const T* Lt_ = h ? Wt : Vt;
        // forward: U(x) chi(x + n mu)
        int cf[4] = {c[0], c[1], c[2], c[3]};
        cf[mu] = (c[mu] + n) % L;
        int cb[4] = {c[0], c[1], c[2], c[3]};
        cb[mu] = ((c[mu] - n) % L + L) % L;
        const long jf = stag_cb(g, cf), jb = stag_cb(g, cb);
        R sf = eta, sb = -eta;
        if (mu == 3) {
          if (c[3] + n >= L) sf *= (R)g.tb;
          if (c[3] - n < 0) sb *= (R)g.tb;
        }
        T vf[3], vb[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
          vf[a] = inr[(long)a * g.stride + jf];
          vb[a] = inr[(long)a * g.stride + jb];
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
          T sfw = {0, 0}, sbw = {0, 0};
#pragma unroll
          for (int b = 0; b < 3; b++) {
            const T uf = Lh[((long)mu * 9 + a * 3 + b) * g.stride + i];   // U(x)_ab
            const T ub = Lt_[((long)mu * 9 + b * 3 + a) * g.stride + jb]; // U(x - n mu)_ba: (U^+)_ab = conj
            const T pf = cm(uf, vf[b]), pb = cmc(ub, vb[b]);
            sfw.x += pf.x;
            sfw.y += pf.y;
            sbw.x += pb.x;
            sbw.y += pb.y;
          }
          acc[a].x += sf * sfw.x + sb * sbw.x;
          acc[a].y += sf * sfw.y + sb * sbw.y;
        }
      }
    }
    T* o = out + r * rhs_stride;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      T v = {alpha * acc[a].x, alpha * acc[a].y};
      if (x) {
        const T xv = x[r * rhs_stride + (long)a * g.stride + i];
        v.x += beta * xv.x;
        v.y += beta * xv.y;
      }
      o[(long)a * g.stride + i] = v;
    }
  }
}

// complex array BLAS (double sums, per-block partials summed on the host in a fixed order)
template <typename T>
__global__ void stag_cdot_kernel(const T* __restrict__ a, const T* __restrict__ b, long n, double* __restrict__ part) {
  double re = 0, im = 0;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const T x = a[k], y = b[k];
    re += (double)x.x * y.x + (double)x.y * y.y;
    im += (double)x.x * y.y - (double)x.y * y.x;
  }
  __shared__ double sh[2][32];
  re = warp_sum(re);
  im = warp_sum(im);
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = re;
    sh[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
      s0 += sh[0][k];
      s1 += sh[1][k];
    }
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}
// y = a x + b y (real a, b)
template <typename T, typename R>
__global__ void stag_axpby_kernel(T* __restrict__ y, const T* __restrict__ x, R a, R b, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const T u = x[k], v = y[k];
    y[k] = {a * u.x + b * v.x, a * u.y + b * v.y};
  }
}
__global__ void stag_to32_kernel(const double2* __restrict__ a, float2* __restrict__ o, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    o[k] = make_float2((float)a[k].x, (float)a[k].y);
}
__global__ void stag_add32_kernel(double2* __restrict__ a, const float2* __restrict__ o, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    a[k] = make_double2(a[k].x + o[k].x, a[k].y + o[k].y);
}

static int sgrid(long n) { return (int)std::max(1L, std::min((n + 127) / 128, 152L * 16)); }

void stag_free(wcl_ctx* c) {
  StagState* s = static_cast<StagState*>(c->stag);
  if (!s) return;
  for (int q = 0; q < 2; q++)
    for (int p = 0; p < 2; p++) {
      cudaFree(s->V[q][p]);
      cudaFree(s->W[q][p]);
    }
  cudaFree(s->part);
  delete s;
  c->stag = nullptr;
}

namespace {

struct Stag {
  wcl_ctx* c;
  StagState* s;
  long half() const { return 3 * s->g.stride; }  // complex numbers per parity field
  // out(parity p) = alpha D in + beta x, precision R
  template <typename R>
  wcl_status dslash(int p, const void* in, const void* x, void* out, double alpha, double beta, int nrhs = 1,
                    long rhs_stride = 0) {
    using T = typename V2<R>::T;
    const int q = std::is_same<R, double>::value ? 0 : 1;
    stag_dslash_kernel<R><<<sgrid((long)nrhs * s->g.vh), 128, 0, c->stream>>>(
        s->g, p, (const T*)s->V[q][0], (const T*)s->V[q][1], (const T*)s->W[q][0], (const T*)s->W[q][1],
        (const T*)in, (const T*)x, (T*)out, (R)alpha, (R)beta, nrhs, rhs_stride);
    WCL_CUDA(cudaGetLastError());
    count_launch(c, true);
    return WCL_OK;
  }
  template <typename T>
  wcl_status dot(const T* a, const T* b, long n, double2* out) {
    const int gb = std::min(STAG_PART, sgrid(n));
    stag_cdot_kernel<T><<<gb, 256, 0, c->stream>>>(a, b, n, s->part);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    WCL_CUDA(cudaMemcpyAsync(s->hpart.data(), s->part, sizeof(double) * 2 * gb, cudaMemcpyDeviceToHost, c->stream));
    WCL_CUDA(cudaStreamSynchronize(c->stream));
    double re = 0, im = 0;
    for (int k = 0; k < gb; k++) {
      re += s->hpart[2 * k];
      im += s->hpart[2 * k + 1];
    }
    *out = make_double2(re, im);
    return WCL_OK;
  }
  template <typename T, typename R>
  wcl_status axpby(T* y, const T* x, double a, double b, long n) {
    stag_axpby_kernel<T, R><<<sgrid(n), 128, 0, c->stream>>>(y, x, (R)a, (R)b, n);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    return WCL_OK;
  }
  // y = M x on the whole lattice (x, y: full fields [2][3][stride])
  template <typename R>
  wcl_status apply_M(void* y, const void* x, int nrhs = 1, long rhs_stride = 0) {
    using T = typename V2<R>::T;
    const T* xe = (const T*)x;
    const T* xo = xe + half();
    T* ye = (T*)y;
    T* yo = ye + half();
    const double m2 = 2 * s->mass;
    WCL_CHECK((dslash<R>(0, xo, xe, ye, 1.0, m2, nrhs, rhs_stride)));
    WCL_CHECK((dslash<R>(1, xe, xo, yo, 1.0, m2, nrhs, rhs_stride)));
    return WCL_OK;
  }
  // FP32 CG on (4 m^2 - D_eo D_oe) e_e = 2 m r_e - D_eo r_o, then e_o = (r_o - D_oe e_e) / (2 m);
  // r, e: full FP32 fields; stops at `target` relative residual of the even system
  wcl_status cg32(float2* e, const float2* r, float2* w, double target, int maxiter, int* iters) {
    const long h = half();
    const double m = s->mass;
    float2 *rhs = w, *res = w + h, *pp = w + 2 * h, *q = w + 3 * h, *t = w + 4 * h;
    // rhs = 2 m r_e - D_eo r_o
    WCL_CHECK((dslash<float>(0, r + h, r, rhs, -1.0, 2 * m)));
    WCL_CUDA(cudaMemsetAsync(e, 0, sizeof(float2) * h, c->stream));
    WCL_CUDA(cudaMemcpyAsync(res, rhs, sizeof(float2) * h, cudaMemcpyDeviceToDevice, c->stream));
    WCL_CUDA(cudaMemcpyAsync(pp, rhs, sizeof(float2) * h, cudaMemcpyDeviceToDevice, c->stream));
    double2 rr;
    WCL_CHECK(dot(res, res, h, &rr));
    const double stop2 = target * target * rr.x;
    int it = 0;
    while (rr.x > stop2 && it < maxiter) {
      // q = 4 m^2 p - D_eo D_oe p
      WCL_CHECK((dslash<float>(1, pp, nullptr, t, 1.0, 0.0)));
      WCL_CHECK((dslash<float>(0, t, pp, q, -1.0, 4 * m * m)));
      double2 pq;
      WCL_CHECK(dot(pp, q, h, &pq));
      if (!(pq.x > 0)) break;
      const double al = rr.x / pq.x;
      WCL_CHECK((axpby<float2, float>(e, pp, al, 1.0, h)));
      WCL_CHECK((axpby<float2, float>(res, q, -al, 1.0, h)));
      double2 rn;
      WCL_CHECK(dot(res, res, h, &rn));
      const double be = rn.x / rr.x;
      rr = rn;
      WCL_CHECK((axpby<float2, float>(pp, res, 1.0, be, h)));
      it++;
    }
    // e_o = (r_o - D_oe e_e) / (2 m)
    WCL_CHECK((dslash<float>(1, e, r + h, e + h, -1.0 / (2 * m), 1.0 / (2 * m))));
    *iters = it;
    return WCL_OK;
  }
};

wcl_status stag_ready(wcl_ctx* c, const char* what) {
  if (!c) return WCL_ERR_INVALID_ARG;
  StagState* s = static_cast<StagState*>(c->stag);
  if (!s || !s->loaded) {
    set_error("%s: no staggered links loaded (wcl_load_staggered)", what);
    return WCL_ERR_NO_GAUGE;
  }
  return WCL_OK;
}

}  // namespace
}  // namespace wcl

using namespace wcl;

extern "C" {

wcl_status wcl_load_staggered(wcl_ctx* c, const void* d_fat, const void* d_long, double mass) {
  if (!c || !d_fat || !d_long) {
    set_error("wcl_load_staggered: null pointer");
    return WCL_ERR_INVALID_ARG;
  }
  if (!(mass > 0) || !std::isfinite(mass)) {
    set_error("wcl_load_staggered: the even-odd solve needs a finite mass > 0");
    return WCL_ERR_INVALID_ARG;
  }
  const void* fat = nullptr;
  const void* lng = nullptr;
  if (!wcl_resolve_field(c, d_fat, &fat, "wcl_load_staggered fat") ||
      !wcl_resolve_field(c, d_long, &lng, "wcl_load_staggered long"))
    return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  StagState* s = static_cast<StagState*>(c->stag);
  if (!s) {
    s = new (std::nothrow) StagState;
    if (!s) return wcl_leave(c, WCL_ERR_OOM);
    c->stag = s;
    s->hpart.assign(2 * STAG_PART, 0.0);
    const size_t b64 = sizeof(double2) * 4 * 9 * c->lat.stride, b32 = sizeof(float2) * 4 * 9 * c->lat.stride;
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < 2 && e == cudaSuccess; p++) {
      e = cudaMalloc(&s->V[0][p], b64);
      if (e == cudaSuccess) e = cudaMalloc(&s->W[0][p], b64);
      if (e == cudaSuccess) e = cudaMalloc(&s->V[1][p], b32);
      if (e == cudaSuccess) e = cudaMalloc(&s->W[1][p], b32);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->V[0][p], 0, b64, c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->W[0][p], 0, b64, c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->V[1][p], 0, b32, c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(s->W[1][p], 0, b32, c->stream);
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->part, sizeof(double) * 2 * STAG_PART);
    if (e != cudaSuccess) {
      stag_free(c);
      return wcl_leave(c, cuda_fail(e, "wcl_load_staggered: allocation"));
    }
  }
  s->loaded = false;
  StagGeom& g = s->g;
  for (int d = 0; d < 4; d++) g.dims[d] = c->lat.dims[d];
  g.lxh = g.dims[0] / 2;
  g.vh = c->lat.vh;
  g.stride = c->lat.stride;
  g.tb = c->lat.tb;
  g.tb_f = (float)c->lat.tb;
  s->mass = mass;
  WCL_CUDA(cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  const long n = 4 * 2 * g.vh * 9;
  stag_links_kernel<<<sgrid(n), 128, 0, c->stream>>>(static_cast<const double2*>(fat), g,
                                                     static_cast<double2*>(s->V[0][0]), static_cast<double2*>(s->V[0][1]),
                                                     static_cast<float2*>(s->V[1][0]), static_cast<float2*>(s->V[1][1]),
                                                     c->d_flags);
  stag_links_kernel<<<sgrid(n), 128, 0, c->stream>>>(static_cast<const double2*>(lng), g,
                                                     static_cast<double2*>(s->W[0][0]), static_cast<double2*>(s->W[0][1]),
                                                     static_cast<float2*>(s->W[1][0]), static_cast<float2*>(s->W[1][1]),
                                                     c->d_flags);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  count_launch(c);
  WCL_CUDA(cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  WCL_CHECK(wcl_leave(c, WCL_OK));
  if (*c->h_flags & 1) {
    set_error("wcl_load_staggered: non-finite link entry");
    return WCL_ERR_NONFINITE;
  }
  s->loaded = true;
  return WCL_OK;
}

wcl_status wcl_apply_staggered(wcl_ctx* c, void* d_out, const void* d_in, wcl_prec prec, int nrhs) {
  WCL_CHECK(stag_ready(c, "wcl_apply_staggered"));
  if (!d_out || !d_in || nrhs < 1 || (prec != WCL_F64 && prec != WCL_F32)) {
    set_error("wcl_apply_staggered: invalid argument (precision F64 or F32, nrhs >= 1)");
    return WCL_ERR_INVALID_ARG;
  }
  const void* in = nullptr;
  const void* outc = nullptr;
  if (!wcl_resolve_field(c, d_in, &in, "wcl_apply_staggered in") ||
      !wcl_resolve_field(c, d_out, &outc, "wcl_apply_staggered out"))
    return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  StagState* s = static_cast<StagState*>(c->stag);
  Stag k{c, s};
  const StagGeom& g = s->g;
  const long full = 2 * k.half();
  std::vector<wcl_ctx*> v{c};
  void *a64 = nullptr, *b64 = nullptr, *a32 = nullptr;
  WCL_CHECK(ws_get(c, "stag_a64", sizeof(double2) * full * nrhs, &a64));
  WCL_CHECK(ws_get(c, "stag_b64", sizeof(double2) * full * nrhs, &b64));
  if (prec == WCL_F32) WCL_CHECK(ws_get(c, "stag_a32", sizeof(float2) * full * 2 * nrhs, &a32));
  WCL_CUDA(cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  const long qdp = 2 * g.vh * 3;
  for (int r = 0; r < nrhs; r++) {
    stag_import_kernel<<<sgrid(qdp), 128, 0, c->stream>>>(static_cast<const double2*>(in) + r * qdp, g,
                                                          static_cast<double2*>(a64) + r * full, c->d_flags);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
  }
  if (prec == WCL_F64) {
    WCL_CHECK(k.apply_M<double>(b64, a64, nrhs, full));
  } else {
    float2* x32 = static_cast<float2*>(a32);
    float2* y32 = x32 + full * nrhs;
    stag_to32_kernel<<<sgrid(full * nrhs), 128, 0, c->stream>>>(static_cast<const double2*>(a64), x32, full * nrhs);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    WCL_CHECK(k.apply_M<float>(y32, x32, nrhs, full));
    WCL_CUDA(cudaMemsetAsync(b64, 0, sizeof(double2) * full * nrhs, c->stream));
    stag_add32_kernel<<<sgrid(full * nrhs), 128, 0, c->stream>>>(static_cast<double2*>(b64), y32, full * nrhs);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
  }
  for (int r = 0; r < nrhs; r++) {
    stag_export_kernel<<<sgrid(qdp), 128, 0, c->stream>>>(static_cast<const double2*>(b64) + r * full, g,
                                                          static_cast<double2*>(const_cast<void*>(outc)) + r * qdp);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
  }
  WCL_CUDA(cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  WCL_CHECK(wcl_leave(c, WCL_OK));
  if (*c->h_flags & 1) {
    set_error("wcl_apply_staggered: non-finite input");
    return WCL_ERR_NONFINITE;
  }
  return WCL_OK;
}

wcl_status wcl_invert_staggered(wcl_ctx* c, void* d_x, const void* d_b, int nrhs, const wcl_solve_params* prm,
                                wcl_solve_info* info) {
  WCL_CHECK(stag_ready(c, "wcl_invert_staggered"));
  if (!d_x || !d_b || !prm || !info || nrhs < 1 || !(prm->tol > 0) || prm->maxiter < 1 ||
      (prm->sloppy != WCL_F32 && prm->sloppy != WCL_F64)) {
    set_error("wcl_invert_staggered: invalid argument (tol > 0, maxiter >= 1, sloppy F32 or F64)");
    return WCL_ERR_INVALID_ARG;
  }
  const void* bp = nullptr;
  const void* xc = nullptr;
  if (!wcl_resolve_field(c, d_b, &bp, "wcl_invert_staggered b") ||
      !wcl_resolve_field(c, d_x, &xc, "wcl_invert_staggered x"))
    return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  const auto t0 = std::chrono::steady_clock::now();
  StagState* s = static_cast<StagState*>(c->stag);
  Stag k{c, s};
  const StagGeom& g = s->g;
  const long h = k.half(), full = 2 * h, qdp = 2 * g.vh * 3;
  void *b64, *x64, *r64, *y64, *w32;
  WCL_CHECK(ws_get(c, "stag_b64", sizeof(double2) * full, &b64));
  WCL_CHECK(ws_get(c, "stag_x64", sizeof(double2) * full, &x64));
  WCL_CHECK(ws_get(c, "stag_r64", sizeof(double2) * full, &r64));
  WCL_CHECK(ws_get(c, "stag_y64", sizeof(double2) * full, &y64));
  WCL_CHECK(ws_get(c, "stag_w32", sizeof(float2) * (2 * full + 5 * h), &w32));
  double2 *B = (double2*)b64, *X = (double2*)x64, *Rr = (double2*)r64, *Y = (double2*)y64;
  float2* r32 = (float2*)w32;
  float2* e32 = r32 + full;
  float2* cgw = e32 + full;
  wcl_status worst = WCL_OK;
  const bool pure64 = prm->sloppy == WCL_F64;
  for (int rhs = 0; rhs < nrhs; rhs++) {
    WCL_CUDA(cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
    stag_import_kernel<<<sgrid(qdp), 128, 0, c->stream>>>(static_cast<const double2*>(bp) + rhs * qdp, g, B,
                                                          c->d_flags);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    double2 bb;
    WCL_CHECK(k.dot(B, B, full, &bb));
    wcl_solve_info& inf = info[rhs];
    inf.iters = 0;
    inf.reliable_updates = 0;
    inf.status = WCL_OK;
    WCL_CUDA(cudaMemsetAsync(X, 0, sizeof(double2) * full, c->stream));
    WCL_CUDA(cudaMemcpyAsync(Rr, B, sizeof(double2) * full, cudaMemcpyDeviceToDevice, c->stream));
    double r2 = bb.x;
    if (!(bb.x == bb.x)) inf.status = WCL_ERR_NONFINITE;
    while (inf.status == WCL_OK && bb.x > 0 && r2 > prm->tol * prm->tol * bb.x) {
      if (inf.iters >= prm->maxiter || inf.reliable_updates > 50) {
        inf.status = WCL_ERR_NOT_CONVERGED;
        break;
      }
      int it = 0;
      if (pure64) {
        // FP64 CG on the even system and the odd reconstruction, in place on double fields
        double2 *rhs = (double2*)y64;  // scratch: reuse y64 halves and cgw as double storage
        void* dw = nullptr;
        WCL_CHECK(ws_get(c, "stag_cg64", sizeof(double2) * 5 * h, &dw));
        double2 *res = (double2*)dw, *pp = res + h, *q = res + 2 * h, *t = res + 3 * h, *e = res + 4 * h;
        const double m = s->mass;
        WCL_CHECK((k.dslash<double>(0, Rr + h, Rr, rhs, -1.0, 2 * m)));
        WCL_CUDA(cudaMemsetAsync(e, 0, sizeof(double2) * h, c->stream));
        WCL_CUDA(cudaMemcpyAsync(res, rhs, sizeof(double2) * h, cudaMemcpyDeviceToDevice, c->stream));
        WCL_CUDA(cudaMemcpyAsync(pp, rhs, sizeof(double2) * h, cudaMemcpyDeviceToDevice, c->stream));
        double2 rr;
        WCL_CHECK(k.dot(res, res, h, &rr));
        const double target = 0.5 * prm->tol * std::sqrt(bb.x / r2);
        const double stop2 = target * target * rr.x;
        while (rr.x > stop2 && inf.iters + it < prm->maxiter) {
          WCL_CHECK((k.dslash<double>(1, pp, nullptr, t, 1.0, 0.0)));
          WCL_CHECK((k.dslash<double>(0, t, pp, q, -1.0, 4 * m * m)));
          double2 pq;
          WCL_CHECK(k.dot(pp, q, h, &pq));
          if (!(pq.x > 0)) break;
          const double al = rr.x / pq.x;
          WCL_CHECK((k.axpby<double2, double>(e, pp, al, 1.0, h)));
          WCL_CHECK((k.axpby<double2, double>(res, q, -al, 1.0, h)));
          double2 rn;
          WCL_CHECK(k.dot(res, res, h, &rn));
          const double be = rn.x / rr.x;
          rr = rn;
          WCL_CHECK((k.axpby<double2, double>(pp, res, 1.0, be, h)));
          it++;
        }
        // x_e += e; x_o += (r_o - D_oe e) / (2 m)
        WCL_CHECK((k.axpby<double2, double>(X, e, 1.0, 1.0, h)));
        WCL_CHECK((k.dslash<double>(1, e, Rr + h, t, -1.0 / (2 * m), 1.0 / (2 * m))));
        WCL_CHECK((k.axpby<double2, double>(X + h, t, 1.0, 1.0, h)));
      } else {
        stag_to32_kernel<<<sgrid(full), 128, 0, c->stream>>>(Rr, r32, full);
        WCL_CUDA(cudaGetLastError());
        count_launch(c);
        const double target = std::max(0.5 * prm->tol * std::sqrt(bb.x / r2), 1e-6);
        WCL_CHECK(k.cg32(e32, r32, cgw, target, prm->maxiter - inf.iters, &it));
        stag_add32_kernel<<<sgrid(full), 128, 0, c->stream>>>(X, e32, full);
        WCL_CUDA(cudaGetLastError());
        count_launch(c);
      }
      inf.iters += it;
      // the true residual of the whole system in FP64
      WCL_CHECK(k.apply_M<double>(Y, X));
      WCL_CHECK((k.axpby<double2, double>(Y, B, 1.0, -1.0, full)));  // Y = B - M X
      WCL_CUDA(cudaMemcpyAsync(Rr, Y, sizeof(double2) * full, cudaMemcpyDeviceToDevice, c->stream));
      double2 rr2;
      WCL_CHECK(k.dot(Rr, Rr, full, &rr2));
      r2 = rr2.x;
      inf.reliable_updates++;
      if (!(r2 == r2)) inf.status = WCL_ERR_NONFINITE;
      if (it == 0 && r2 > prm->tol * prm->tol * bb.x) inf.status = WCL_ERR_BREAKDOWN;
    }
    inf.true_residual = bb.x > 0 ? std::sqrt(r2 / bb.x) : 0.0;
    stag_export_kernel<<<sgrid(qdp), 128, 0, c->stream>>>(X, g, static_cast<double2*>(const_cast<void*>(xc)) + rhs * qdp);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    WCL_CUDA(cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    WCL_CUDA(cudaStreamSynchronize(c->stream));
    if (*c->h_flags & 1) inf.status = WCL_ERR_NONFINITE;
    if (worst == WCL_OK && inf.status != WCL_OK) worst = (wcl_status)inf.status;
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int r = 0; r < nrhs; r++) info[r].seconds = secs;
  if (worst != WCL_OK) set_error("wcl_invert_staggered: a right-hand side did not reach the tolerance");
  return wcl_leave(c, worst);
}

}  // extern "C"
