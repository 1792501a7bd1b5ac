// HISQ link smearing: the fat and long links of the staggered operator (stag.cu) built
// from the thin gauge links, in FP64.
//
// Sec. II.A names the HISQ process (Follana et al.) in the MILC convention: a first
// fattening step, a U(3) projection of its result, a second fattening step with the
// Naik term.  A smearing with coefficients (c1, c3, c5, c7, cL) replaces each link by
//   c1 U_mu + c3 sum S3 + c5 sum S5 + c7 sum S7 + cL sum SL,
// where staple(+-rho, F) carries a mu-directed object F one step along +-rho and back,
//   staple(+rho, F)(x) = U_rho(x) F(x + rho) U_rho(x + mu)^+,
//   staple(-rho, F)(x) = U_rho(x - rho)^+ F(x - rho) U_rho(x - rho + mu),
// S3 = staple(r, U_mu), S5 = staple(r, staple(s, U_mu)) and S7 = staple(r, staple(s,
// staple(n, U_mu))) over signed directions on different axes (all orderings), and the
// Lepage term SL = staple(r, staple(r, U_mu)) (the straight 5-link staple).
//   first level:  (1/8, 1/16, 1/64, 1/384, 0): fat7, the expansion of
//                 prod_{rho != mu} (1 + delta_rho^2 / 4);
//   projection:   W = V (V^+ V)^(-1/2) (U(3), the unitary polar factor);
//   second level: (5/8, 1/16, 1/64, 1/384, -1/16) on W, plus eps/8 W; long links
//                 -(1 + eps)/24 W_mu(x) W_mu(x + mu) W_mu(x + 2 mu).
// A staple is linear in F, so the sums are built from the inside out, one staple pass
// (one kernel launch over the lattice, both signs) per term:
//   T1 = c5 U_mu + c7 sum_{+-nu} staple(nu, U_mu)          nu: the fourth axis
//   T2 = c3 U_mu + sum_{sigma} sum_{+-sigma} staple(sigma, T1)
//   out_mu = c1 U_mu + sum_{rho} sum_{+-rho} staple(rho, T2) + cL sum staple(rho, staple(rho, U_mu)).
// (V^+ V)^(-1/2) = f0 + f1 Q + f2 Q^2 with Q = V^+ V (Cayley-Hamilton): with s_k the
// square roots of Q's eigenvalues, u = sum s_k, v = sum_{j<k} s_j s_k, w = prod s_k,
// the quadratic through (lambda_k, lambda_k^(-1/2)) has f2 = u / d, f1 = (2 u v - w - u^3) / d,
// f0 = (u v^2 - w (u^2 + v)) / d, d = w (u v - w).  The eigenvalues of the Hermitian 3x3
// Q come from the trigonometric solution of its characteristic cubic (O. K. Smith,
// Comm. ACM 4 (1961) 168).
//
// Layouts: caller links are the QDP gauge layout [4][2][Lt][Lz][Ly][Lx/2][3][3]
// complex128; internally every link field is lexicographic [mu][site][9] double2 over
// the whole lattice (site = ((t Lz + z) Ly + y) Lx + x), one thread per site.
#include <algorithm>
#include <cmath>

#include "context.cuh"

wcl_status wcl_enter(wcl_ctx* c);
wcl_status wcl_leave(wcl_ctx* c, wcl_status s);
bool wcl_resolve_field(const wcl_ctx* c, const void* p, const void** out, const char* what);

namespace wcl {
namespace {

constexpr int HISQ_NONFINITE = 1, HISQ_SINGULAR = 8;  // bits of the context's error word

struct HGeom {
  int d[4];
  long v;  // sites
};

struct M3 {
  double2 e[9];
};

__device__ __forceinline__ double2 hmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 hmulc(double2 a, double2 b) {  // a conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 hcmul(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 hadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 hscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

__device__ __forceinline__ void mload(M3& m, const double2* f, long s) {
#pragma unroll
  for (int k = 0; k < 9; k++) m.e[k] = f[s * 9 + k];
}
// a b
__device__ __forceinline__ M3 mmul(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; k++) acc = hadd(acc, hmul(a.e[3 * i + k], b.e[3 * k + j]));
      r.e[3 * i + j] = acc;
    }
  return r;
}
// a b^+
__device__ __forceinline__ M3 mmul_nd(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; k++) acc = hadd(acc, hmulc(a.e[3 * i + k], b.e[3 * j + k]));
      r.e[3 * i + j] = acc;
    }
  return r;
}
// a^+ b
__device__ __forceinline__ M3 mmul_dn(const M3& a, const M3& b) {
  M3 r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      double2 acc = make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; k++) acc = hadd(acc, hcmul(a.e[3 * k + i], b.e[3 * k + j]));
      r.e[3 * i + j] = acc;
    }
  return r;
}

__device__ __forceinline__ void coords(const HGeom& g, long s, int c[4]) {
  c[0] = (int)(s % g.d[0]);
  long q = s / g.d[0];
  c[1] = (int)(q % g.d[1]);
  q /= g.d[1];
  c[2] = (int)(q % g.d[2]);
  c[3] = (int)(q / g.d[2]);
}
__device__ __forceinline__ long site_of(const HGeom& g, const int c[4]) {
  return (((long)c[3] * g.d[2] + c[2]) * g.d[1] + c[1]) * g.d[0] + c[0];
}
// the site n steps along mu from coordinates c (periodic)
__device__ __forceinline__ long hop(const HGeom& g, const int c[4], int mu, int n) {
  int cc[4] = {c[0], c[1], c[2], c[3]};
  cc[mu] = ((cc[mu] + n) % g.d[mu] + g.d[mu]) % g.d[mu];
  return site_of(g, cc);
}

// QDP cb2 links -> lexicographic [mu][site][9]; a non-finite entry sets HISQ_NONFINITE
__global__ void hisq_import_kernel(const double2* __restrict__ qdp, double2* __restrict__ U, HGeom g,
                                   int* flags) {
  const long n = 4 * g.v;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(e / g.v);
    const long s = e - mu * g.v;
    int c[4];
    coords(g, s, c);
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    const long vh = g.v / 2;
    const long i = (((long)c[3] * g.d[2] + c[2]) * g.d[1] + c[1]) * (g.d[0] / 2) + c[0] / 2;
    const double2* src = qdp + (((long)mu * 2 + p) * vh + i) * 9;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const double2 v = src[k];
      bad |= !isfinite(v.x) || !isfinite(v.y);
      U[e * 9 + k] = v;
    }
    if (bad) atomicOr(flags, HISQ_NONFINITE);
  }
}

// lexicographic [mu][site][9] -> QDP cb2 links
__global__ void hisq_export_kernel(const double2* __restrict__ U, double2* __restrict__ qdp, HGeom g) {
  const long n = 4 * g.v;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(e / g.v);
    const long s = e - mu * g.v;
    int c[4];
    coords(g, s, c);
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    const long vh = g.v / 2;
    const long i = (((long)c[3] * g.d[2] + c[2]) * g.d[1] + c[1]) * (g.d[0] / 2) + c[0] / 2;
    double2* dst = qdp + (((long)mu * 2 + p) * vh + i) * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) dst[k] = U[e * 9 + k];
  }
}

// out = a X + b Y over n complex entries (Y may be null; out may be X)
__global__ void hisq_lin_kernel(double2* out, double a, const double2* X, double b, const double2* Y, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    double2 v = hscale(a, X[e]);
    if (Y) v = hadd(v, hscale(b, Y[e]));
    out[e] = v;
  }
}

// out(x) = alpha out(x) + beta sum_{signs} staple(+-rho, F)(x) for the mu-directed field F;
// signs: bit 0 the +rho staple, bit 1 the -rho staple; U the links [mu][site][9]
__global__ void hisq_staple_kernel(const double2* __restrict__ U, const double2* __restrict__ F,
                                   double2* __restrict__ out, HGeom g, int mu, int rho, int signs, double alpha,
                                   double beta) {
  const double2* Ur = U + (long)rho * g.v * 9;
  for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < g.v; s += (long)gridDim.x * blockDim.x) {
    int c[4];
    coords(g, s, c);
    M3 acc;
#pragma unroll
    for (int k = 0; k < 9; k++) acc.e[k] = make_double2(0.0, 0.0);
    if (signs & 1) {
      M3 a, f, b;
      mload(a, Ur, s);                     // U_rho(x)
      mload(f, F, hop(g, c, rho, 1));      // F(x + rho)
      mload(b, Ur, hop(g, c, mu, 1));      // U_rho(x + mu)
      const M3 t = mmul_nd(mmul(a, f), b);
#pragma unroll
      for (int k = 0; k < 9; k++) acc.e[k] = hadd(acc.e[k], t.e[k]);
    }
    if (signs & 2) {
      const long xb = hop(g, c, rho, -1);
      int cb[4] = {c[0], c[1], c[2], c[3]};
      cb[rho] = (cb[rho] - 1 + g.d[rho]) % g.d[rho];
      M3 a, f, b;
      mload(a, Ur, xb);                    // U_rho(x - rho)
      mload(f, F, xb);                     // F(x - rho)
      mload(b, Ur, hop(g, cb, mu, 1));     // U_rho(x - rho + mu)
      const M3 t = mmul(mmul_dn(a, f), b);
#pragma unroll
      for (int k = 0; k < 9; k++) acc.e[k] = hadd(acc.e[k], t.e[k]);
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
      double2 v = hscale(beta, acc.e[k]);
      if (alpha != 0.0) v = hadd(v, hscale(alpha, out[s * 9 + k]));
      out[s * 9 + k] = v;
    }
  }
}

// W = V (V^+ V)^(-1/2); false if V^+ V is not positive definite (or not finite)
__device__ __forceinline__ bool u3_link(const M3& V, M3& W) {
  const M3 Q = mmul_dn(V, V);
  const double q00 = Q.e[0].x, q11 = Q.e[4].x, q22 = Q.e[8].x;
  const double m = (q00 + q11 + q22) / 3.0;
  const double k00 = q00 - m, k11 = q11 - m, k22 = q22 - m;
  const double2 q01 = Q.e[1], q02 = Q.e[2], q12 = Q.e[5];
  const double a01 = q01.x * q01.x + q01.y * q01.y, a02 = q02.x * q02.x + q02.y * q02.y,
               a12 = q12.x * q12.x + q12.y * q12.y;
  // K = Q - m: p = tr(K^2) / 6, q = det(K) / 2
  const double p = (k00 * k00 + k11 * k11 + k22 * k22 + 2.0 * (a01 + a02 + a12)) / 6.0;
  const double2 cyc = hmulc(hmul(q01, q12), q02);  // q01 q12 conj(q02)
  const double q = 0.5 * (k00 * k11 * k22 + 2.0 * cyc.x - k00 * a12 - k11 * a02 - k22 * a01);
  double phi = 0.0;
  if (p > 0.0) {
    const double r = q / (p * sqrt(p));
    phi = acos(fmin(1.0, fmax(-1.0, r))) / 3.0;
  }
  const double sp = 2.0 * sqrt(p), third = 2.0943951023931954923;  // 2 pi / 3
  const double l0 = m + sp * cos(phi), l1 = m + sp * cos(phi + third), l2 = m + sp * cos(phi + 2.0 * third);
  const double lmin = fmin(l0, fmin(l1, l2));
  if (!(lmin > 1e-12 * m) || !isfinite(m)) return false;
  const double s0 = sqrt(l0), s1 = sqrt(l1), s2 = sqrt(l2);
  const double u = s0 + s1 + s2, v = s0 * s1 + s0 * s2 + s1 * s2, w = s0 * s1 * s2;
  const double den = w * (u * v - w);
  const double f0 = (u * v * v - w * (u * u + v)) / den, f1 = (2.0 * u * v - w - u * u * u) / den, f2 = u / den;
  const M3 Q2 = mmul(Q, Q);
  M3 R;
#pragma unroll
  for (int k = 0; k < 9; k++) R.e[k] = hadd(hscale(f1, Q.e[k]), hscale(f2, Q2.e[k]));
#pragma unroll
  for (int k = 0; k < 9; k += 4) R.e[k].x += f0;
  W = mmul(V, R);
  return true;
}

__global__ void hisq_u3_kernel(double2* __restrict__ V, long nlinks, int* flags) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nlinks; e += (long)gridDim.x * blockDim.x) {
    M3 a, w;
    mload(a, V, e);
    if (!u3_link(a, w)) {
      atomicOr(flags, HISQ_SINGULAR);
#pragma unroll
      for (int k = 0; k < 9; k++) w.e[k] = make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int k = 0; k < 9; k++) V[e * 9 + k] = w.e[k];
  }
}

// N_mu(x) = coeff W_mu(x) W_mu(x + mu) W_mu(x + 2 mu)
__global__ void hisq_naik_kernel(const double2* __restrict__ W, double2* __restrict__ N, HGeom g, double coeff) {
  const long n = 4 * g.v;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(e / g.v);
    const long s = e - mu * g.v;
    const double2* Wm = W + (long)mu * g.v * 9;
    int c[4];
    coords(g, s, c);
    M3 a, b, d;
    mload(a, Wm, s);
    mload(b, Wm, hop(g, c, mu, 1));
    mload(d, Wm, hop(g, c, mu, 2));
    const M3 r = mmul(mmul(a, b), d);
#pragma unroll
    for (int k = 0; k < 9; k++) N[e * 9 + k] = hscale(coeff, r.e[k]);
  }
}

int hgrid(long n) { return (int)std::max(1L, std::min((n + 127) / 128, 152L * 32)); }

struct HisqRun {
  wcl_ctx* c;
  HGeom g;
  long f;  // complex entries of one mu-directed field
  cudaError_t lin(double2* out, double a, const double2* X, double b = 0.0, const double2* Y = nullptr) {
    hisq_lin_kernel<<<hgrid(f), 128, 0, c->stream>>>(out, a, X, b, Y, f);
    count_launch(c);
    return cudaGetLastError();
  }
  cudaError_t staple(const double2* U, double2* out, const double2* F, int mu, int rho, int signs, double alpha,
                     double beta) {
    hisq_staple_kernel<<<hgrid(g.v), 128, 0, c->stream>>>(U, F, out, g, mu, rho, signs, alpha, beta);
    count_launch(c);
    return cudaGetLastError();
  }
  // D = the smearing of the link set S with coefficients (c1, c3, c5, c7, cL)
  cudaError_t level(const double2* S, double2* D, double2* T1, double2* T2, double2* T3, const double cf[5]) {
    cudaError_t e = cudaSuccess;
    for (int mu = 0; mu < 4 && e == cudaSuccess; mu++) {
      const double2* Sm = S + mu * f;
      double2* Dm = D + mu * f;
      e = lin(Dm, cf[0], Sm);
      for (int rho = 0; rho < 4 && e == cudaSuccess; rho++) {
        if (rho == mu) continue;
        e = lin(T2, cf[1], Sm);
        for (int sig = 0; sig < 4 && e == cudaSuccess; sig++) {
          if (sig == mu || sig == rho) continue;
          const int nu = 6 - mu - rho - sig;
          e = lin(T1, cf[2], Sm);
          if (e == cudaSuccess) e = staple(S, T1, Sm, mu, nu, 3, 1.0, cf[3]);
          if (e == cudaSuccess) e = staple(S, T2, T1, mu, sig, 3, 1.0, 1.0);
        }
        if (e == cudaSuccess) e = staple(S, Dm, T2, mu, rho, 3, 1.0, 1.0);
        if (cf[4] != 0.0)
          for (int sign = 1; sign <= 2 && e == cudaSuccess; sign++) {
            e = staple(S, T3, Sm, mu, rho, sign, 0.0, 1.0);
            if (e == cudaSuccess) e = staple(S, Dm, T3, mu, rho, sign, 1.0, cf[4]);
          }
      }
    }
    return e;
  }
};

}  // namespace
}  // namespace wcl

using namespace wcl;

extern "C" {

wcl_status wcl_hisq_smear(wcl_ctx* c, void* d_fat, void* d_long, const void* d_gauge, double eps_naik) {
  if (!c || !d_fat || !d_long || !d_gauge || !std::isfinite(eps_naik)) {
    set_error("wcl_hisq_smear: null pointer or non-finite eps_naik");
    return WCL_ERR_INVALID_ARG;
  }
  const void *gin = nullptr, *fo = nullptr, *lo = nullptr;
  if (!wcl_resolve_field(c, d_gauge, &gin, "wcl_hisq_smear gauge") ||
      !wcl_resolve_field(c, d_fat, &fo, "wcl_hisq_smear fat") ||
      !wcl_resolve_field(c, d_long, &lo, "wcl_hisq_smear long"))
    return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  HisqRun r;
  r.c = c;
  for (int d = 0; d < 4; d++) r.g.d[d] = c->lat.dims[d];
  r.g.v = 2 * c->lat.vh;
  r.f = r.g.v * 9;
  // thin links (later the Naik links), first level / projected links, second level, 3 temporaries
  double2* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(double2) * (size_t)r.f * 15);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("wcl_hisq_smear: cannot allocate %zu bytes", sizeof(double2) * (size_t)r.f * 15);
    return wcl_leave(c, WCL_ERR_OOM);
  }
  double2 *U = buf, *V = buf + 4 * r.f, *X = buf + 8 * r.f, *T1 = buf + 12 * r.f, *T2 = buf + 13 * r.f,
          *T3 = buf + 14 * r.f;
  static const double fat7[5] = {1.0 / 8, 1.0 / 16, 1.0 / 64, 1.0 / 384, 0.0};
  static const double asq[5] = {5.0 / 8, 1.0 / 16, 1.0 / 64, 1.0 / 384, -1.0 / 16};
  e = cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) {
    hisq_import_kernel<<<hgrid(4 * r.g.v), 128, 0, c->stream>>>(static_cast<const double2*>(gin), U, r.g, c->d_flags);
    count_launch(c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = r.level(U, V, T1, T2, T3, fat7);
  if (e == cudaSuccess) {
    hisq_u3_kernel<<<hgrid(4 * r.g.v), 128, 0, c->stream>>>(V, 4 * r.g.v, c->d_flags);
    count_launch(c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = r.level(V, X, T1, T2, T3, asq);
  if (e == cudaSuccess && eps_naik != 0.0) {
    hisq_lin_kernel<<<hgrid(4 * r.f), 128, 0, c->stream>>>(X, 1.0, X, eps_naik / 8.0, V, 4 * r.f);
    count_launch(c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    hisq_naik_kernel<<<hgrid(4 * r.g.v), 128, 0, c->stream>>>(V, U, r.g, -(1.0 + eps_naik) / 24.0);
    count_launch(c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    hisq_export_kernel<<<hgrid(4 * r.g.v), 128, 0, c->stream>>>(X, static_cast<double2*>(const_cast<void*>(fo)), r.g);
    hisq_export_kernel<<<hgrid(4 * r.g.v), 128, 0, c->stream>>>(U, static_cast<double2*>(const_cast<void*>(lo)), r.g);
    count_launch(c);
    count_launch(c);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  if (e != cudaSuccess) return wcl_leave(c, cuda_fail(e, "wcl_hisq_smear"));
  const int fl = c->h_flags[0];
  if (fl & HISQ_NONFINITE) {
    set_error("wcl_hisq_smear: non-finite entry in the thin links");
    return wcl_leave(c, WCL_ERR_NONFINITE);
  }
  if (fl & HISQ_SINGULAR) {
    set_error("wcl_hisq_smear: a first-level fat link V has V^+ V not positive definite (no U(3) projection)");
    return wcl_leave(c, WCL_ERR_RECONSTRUCT);
  }
  return wcl_leave(c, WCL_OK);
}

}  // extern "C"
