// Fused even-odd Wilson hopping term + clover (Eq. 5, isotropic):
//
//   out = C_post ( alpha * D_{p,1-p} in  +  beta * C_pre x )
//
// on output parity p, for every (lattice, rhs) slice of a batch.  D is the
// hopping term H restricted to (out parity p, in parity 1-p):
//   D psi(s) = sum_mu eta (1 - g_mu) U_mu(s) psi(s+mu) + eta (1 + g_mu) U_mu(s-mu)^+ psi(s-mu)
// and with DAG the projector signs are swapped (gamma5 D gamma5 = D^+).
// C_post / C_pre are clover blocks (A or A^-1) of parity p, or absent.
//
// One thread owns one output site.  Per direction the neighbour spinor is
// spin-projected to a half spinor (2 spins x 3 colours), multiplied by the link
// (or its adjoint), and the 4-spinor is rebuilt while accumulating.  The
// DeGrand-Rossi projections, written for (1 + s*gamma_mu):
//   mu=x: h0 = p0 + s i p3, h1 = p1 + s i p2;  rows 2,3 = -s i h1, -s i h0
//   mu=y: h0 = p0 - s p3,   h1 = p1 + s p2;    rows 2,3 =  s h1,  -s h0
//   mu=z: h0 = p0 + s i p2, h1 = p1 - s i p3;  rows 2,3 = -s i h0,  s i h1
//   mu=t: h0 = p0 + s p2,   h1 = p1 + s p3;    rows 2,3 =  s h0,   s h1
#pragma once
#include <algorithm>

#include "blas.cuh"
#include "internal.cuh"

namespace wcl {

// MODE_RECON (with POST, XPAY and PRE): t = alpha D in + beta x, out = C_post t,
// out2 = t - C_pre out.  With C_post = A^-1, C_pre = A this reconstructs the odd
// solution x_o = A_oo^-1 (b_o + kappa D_oe x_e) and its residual b_o - (A x_o - kappa D x_e)
// in one pass over the links.
enum DslashMode { MODE_POST = 1, MODE_XPAY = 2, MODE_PRE = 4, MODE_RECON = 8 };

// Reductions fused into the epilogue of an XPAY launch (the second half of
// M_hat), finalised on the device like the stand-alone reductions:
//   EPI_ALPHA   <f, out>              -> BiCGStab alpha = rho / <rhat, v>     (f = rhat)
//   EPI_OMEGA   <out, x>, ||out||^2   -> BiCGStab omega = <t, s> / <t, t>    (x = s)
//   EPI_CGALPHA ||out||^2             -> CG alpha = zz / ||q||^2
//   EPI_CGZ     ||out||^2             -> CG zz' and beta = zz' / zz
enum DslashEpi { EPI_NONE = 0, EPI_ALPHA = 1, EPI_OMEGA = 2, EPI_CGALPHA = 3, EPI_CGZ = 4 };

struct DslashArgs {
  Batch b;
  FieldRef out, in, x, out2;
  const void* gauge[MAXLAT][2];  // per parity: [mu][chunk][stride]
  const void* cpost[MAXLAT];
  const float* cpost_norm[MAXLAT];
  const void* cpre[MAXLAT];
  const float* cpre_norm[MAXLAT];
  double alpha[MAXLAT], beta[MAXLAT];
  int out_parity;
  const int* active;  // per slot; null = every slice active
  // epilogue reduction
  FieldRef f;
  double* partials;   // [slot][maxch][3]
  unsigned* counters; // [slot], zero between launches
  Scalars* sc;
  int maxch;
  int nrhs_tc;        // tensor-core kernel: right-hand sides per lattice (one CTA covers all)
};

template <int EPI>
__device__ __forceinline__ void epi_finalize(Scalars& c, const double* t) {
  if (EPI == EPI_ALPHA) BicgAlpha<F32>{}.finalize(c, t);
  if (EPI == EPI_OMEGA) BicgOmega<F32>{}.finalize(c, t);
  if (EPI == EPI_CGALPHA) CgAlpha<F32>{}.finalize(c, t);
  if (EPI == EPI_CGZ) CgZnorm<F32>{}.finalize(c, t);
}

template <int MU, int S, typename R>
__device__ __forceinline__ void project(const cpx<R> p[12], cpx<R> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<R> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
    if (MU == 0) {
      h[c] = (S > 0) ? p0 + ti(p3) : p0 - ti(p3);
      h[3 + c] = (S > 0) ? p1 + ti(p2) : p1 - ti(p2);
    } else if (MU == 1) {
      h[c] = (S > 0) ? p0 - p3 : p0 + p3;
      h[3 + c] = (S > 0) ? p1 + p2 : p1 - p2;
    } else if (MU == 2) {
      h[c] = (S > 0) ? p0 + ti(p2) : p0 - ti(p2);
      h[3 + c] = (S > 0) ? p1 - ti(p3) : p1 + ti(p3);
    } else {
      h[c] = (S > 0) ? p0 + p2 : p0 - p2;
      h[3 + c] = (S > 0) ? p1 + p3 : p1 - p3;
    }
  }
}

template <int MU, int S, typename R>
__device__ __forceinline__ void reconstruct_acc(cpx<R> acc[12], const cpx<R> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<R> h0 = h[c], h1 = h[3 + c];
    acc[c] = acc[c] + h0;
    acc[3 + c] = acc[3 + c] + h1;
    if (MU == 0) {
      acc[6 + c] = (S > 0) ? acc[6 + c] - ti(h1) : acc[6 + c] + ti(h1);
      acc[9 + c] = (S > 0) ? acc[9 + c] - ti(h0) : acc[9 + c] + ti(h0);
    } else if (MU == 1) {
      acc[6 + c] = (S > 0) ? acc[6 + c] + h1 : acc[6 + c] - h1;
      acc[9 + c] = (S > 0) ? acc[9 + c] - h0 : acc[9 + c] + h0;
    } else if (MU == 2) {
      acc[6 + c] = (S > 0) ? acc[6 + c] - ti(h0) : acc[6 + c] + ti(h0);
      acc[9 + c] = (S > 0) ? acc[9 + c] + ti(h1) : acc[9 + c] - ti(h1);
    } else {
      acc[6 + c] = (S > 0) ? acc[6 + c] + h0 : acc[6 + c] - h0;
      acc[9 + c] = (S > 0) ? acc[9 + c] + h1 : acc[9 + c] - h1;
    }
  }
}

// uh = U h (ADJ = false) or U^+ h (ADJ = true), for both half-spinor components
template <bool ADJ, typename R>
__device__ __forceinline__ void link_mul(const cpx<R> u[3][3], const cpx<R> h[6], cpx<R> o[6], R sign) {
#pragma unroll
  for (int k = 0; k < 2; k++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cpx<R> acc = {0, 0};
#pragma unroll
      for (int bb = 0; bb < 3; bb++) {
        if (ADJ)
          cfma_conj(acc, u[bb][a], h[3 * k + bb]);
        else
          cfma(acc, u[a][bb], h[3 * k + bb]);
      }
      o[3 * k + a] = sign * acc;
    }
  }
}

template <int P, int MU, bool DAG>
__device__ __forceinline__ void hop_dir(cpx<typename Traits<P>::R> acc[12], const void* in, const float* in_norm,
                                        const void* g_here, const void* g_there, long stride, long i, long jf,
                                        long jb, typename Traits<P>::R sf, typename Traits<P>::R sb) {
  using R = typename Traits<P>::R;
  constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF*gamma
  constexpr int SB = -SF;
  cpx<R> psi[12], h[6], uh[6], u[3][3];
  // forward: U_mu(s) psi(s + mu)
  SpinorIO<P>::load(psi, in, in_norm, stride, jf);
  LinkIO<P>::load(u, g_here, stride, i, MU);
  project<MU, SF>(psi, h);
  link_mul<false>(u, h, uh, sf);
  reconstruct_acc<MU, SF>(acc, uh);
  // backward: U_mu(s - mu)^+ psi(s - mu)
  SpinorIO<P>::load(psi, in, in_norm, stride, jb);
  LinkIO<P>::load(u, g_there, stride, jb, MU);
  project<MU, SB>(psi, h);
  link_mul<true>(u, h, uh, sb);
  reconstruct_acc<MU, SB>(acc, uh);
}

// The hopping term with mu as a loop variable: one copy of the forward and one of
// the adjoint link multiply instead of eight inlined ones.  Used for the
// double-float kernel, whose fully unrolled code overflows the instruction cache
// (ncu: "no instruction" the dominant stall).  With the rolled spin loop of the
// link multiply and one copy of the clover block multiply: 16.1 -> 10.3 ms per
// 12-RHS launch at 32^3x64.
template <int S, typename R>
__device__ __forceinline__ void project_rt(int mu, const cpx<R> p[12], cpx<R> h[6]) {
  switch (mu) {
    case 0: project<0, S>(p, h); break;
    case 1: project<1, S>(p, h); break;
    case 2: project<2, S>(p, h); break;
    default: project<3, S>(p, h); break;
  }
}
template <int S, typename R>
__device__ __forceinline__ void reconstruct_rt(int mu, cpx<R> acc[12], const cpx<R> h[6]) {
  switch (mu) {
    case 0: reconstruct_acc<0, S>(acc, h); break;
    case 1: reconstruct_acc<1, S>(acc, h); break;
    case 2: reconstruct_acc<2, S>(acc, h); break;
    default: reconstruct_acc<3, S>(acc, h); break;
  }
}

// link multiply with the two spin halves as a loop (code size, see hop_all_compact)
template <bool ADJ, typename R>
__device__ __forceinline__ void link_mul_rolled(const cpx<R> u[3][3], const cpx<R> h[6], cpx<R> o[6], R sign) {
#pragma unroll 1
  for (int k = 0; k < 2; k++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cpx<R> acc = {R(0), R(0)};
#pragma unroll
      for (int bb = 0; bb < 3; bb++) {
        if (ADJ)
          cfma_conj(acc, u[bb][a], h[3 * k + bb]);
        else
          cfma(acc, u[a][bb], h[3 * k + bb]);
      }
      o[3 * k + a] = sign * acc;
    }
  }
}

template <int P, bool DAG>
__device__ __forceinline__ void hop_all_compact(cpx<typename Traits<P>::R> acc[12], const void* in, const float* in_norm,
                                             const void* g_here, const void* g_there, long stride, long i,
                                             const long jf[4], const long jb[4], typename Traits<P>::R sf,
                                             typename Traits<P>::R sb) {
  using R = typename Traits<P>::R;
  constexpr int SF = DAG ? +1 : -1;
  constexpr int SB = -SF;
#pragma unroll 1
  for (int mu = 0; mu < 4; mu++) {
    cpx<R> psi[12], h[6], uh[6], u[3][3];
    SpinorIO<P>::load(psi, in, in_norm, stride, jf[mu]);
    LinkIO<P>::load(u, g_here, stride, i, mu);
    project_rt<SF>(mu, psi, h);
    link_mul_rolled<false>(u, h, uh, mu == 3 ? sf : R(1));
    reconstruct_rt<SF>(mu, acc, uh);
    SpinorIO<P>::load(psi, in, in_norm, stride, jb[mu]);
    LinkIO<P>::load(u, g_there, stride, jb[mu], mu);
    project_rt<SB>(mu, psi, h);
    link_mul_rolled<true>(u, h, uh, mu == 3 ? sb : R(1));
    reconstruct_rt<SB>(mu, acc, uh);
  }
}

template <int P, bool DAG, int MODE, int EPI>
__device__ __forceinline__ void dslash_site(const DslashArgs& a, const Slice& s, const LatGeom& g, long i,
                                            double red[3]) {
  using R = typename Traits<P>::R;
  const long stride = g.stride;
  const int p = a.out_parity;

  // coordinates of the output site
  const int lxh = g.lxh, Lx = g.dims[0], Ly = g.dims[1], Lz = g.dims[2], Lt = g.dims[3];
  const int xh = (int)(i % lxh);
  int rem = (int)(i / lxh);
  const int y = rem % Ly;
  rem /= Ly;
  const int z = rem % Lz;
  const int t = rem / Lz;
  const int x = 2 * xh + ((p + y + z + t) & 1);
  const long row = i - xh;
  const long plane = (long)lxh * Ly, vol3 = plane * Lz;

  const void* in = rhs_ptr<P>(a.in, s.l, s.rhs, stride);
  const float* in_norm = rhs_norm(a.in, s.l, s.rhs, stride);
  const void* g_here = a.gauge[s.l][p];
  const void* g_there = a.gauge[s.l][1 - p];

  cpx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {0, 0};

  if constexpr (P == DF64) {
    const long jf[4] = {row + ((x + 1 == Lx ? 0 : x + 1) >> 1), (y + 1 == Ly) ? i - (long)(Ly - 1) * lxh : i + lxh,
                        (z + 1 == Lz) ? i - (long)(Lz - 1) * plane : i + plane,
                        (t + 1 == Lt) ? i - (long)(Lt - 1) * vol3 : i + vol3};
    const long jb[4] = {row + ((x == 0 ? Lx - 1 : x - 1) >> 1), (y == 0) ? i + (long)(Ly - 1) * lxh : i - lxh,
                        (z == 0) ? i + (long)(Lz - 1) * plane : i - plane,
                        (t == 0) ? i + (long)(Lt - 1) * vol3 : i - vol3};
    hop_all_compact<P, DAG>(acc, in, in_norm, g_here, g_there, stride, i, jf, jb,
                            hop_t_weight<R>(g, t + 1 == Lt), hop_t_weight<R>(g, t == 0));
  } else {
  {
    const long jf = row + ((x + 1 == Lx ? 0 : x + 1) >> 1);
    const long jb = row + ((x == 0 ? Lx - 1 : x - 1) >> 1);
    hop_dir<P, 0, DAG>(acc, in, in_norm, g_here, g_there, stride, i, jf, jb, R(1), R(1));
  }
  {
    const long jf = (y + 1 == Ly) ? i - (long)(Ly - 1) * lxh : i + lxh;
    const long jb = (y == 0) ? i + (long)(Ly - 1) * lxh : i - lxh;
    hop_dir<P, 1, DAG>(acc, in, in_norm, g_here, g_there, stride, i, jf, jb, R(1), R(1));
  }
  {
    const long jf = (z + 1 == Lz) ? i - (long)(Lz - 1) * plane : i + plane;
    const long jb = (z == 0) ? i + (long)(Lz - 1) * plane : i - plane;
    hop_dir<P, 2, DAG>(acc, in, in_norm, g_here, g_there, stride, i, jf, jb, R(1), R(1));
  }
  {
    const long jf = (t + 1 == Lt) ? i - (long)(Lt - 1) * vol3 : i + vol3;
    const long jb = (t == 0) ? i + (long)(Lt - 1) * vol3 : i - vol3;
    const R sf = hop_t_weight<R>(g, t + 1 == Lt);
    const R sb = hop_t_weight<R>(g, t == 0);
    hop_dir<P, 3, DAG>(acc, in, in_norm, g_here, g_there, stride, i, jf, jb, sf, sb);
  }
  }

  const R alpha = R(a.alpha[s.l]);
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = alpha * acc[k];

  if (MODE & MODE_RECON) {
    cpx<R> xv[12], y2[12], ay[12];
    SpinorIO<P>::load(xv, rhs_ptr<P>(a.x, s.l, s.rhs, stride), rhs_norm(a.x, s.l, s.rhs, stride), stride, i);
    const R beta = R(a.beta[s.l]);
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = acc[k] + beta * xv[k];
    CloverIO<P>::apply(y2, acc, a.cpost[s.l], a.cpost_norm[s.l], stride, i);
    CloverIO<P>::apply(ay, y2, a.cpre[s.l], a.cpre_norm[s.l], stride, i);
#pragma unroll
    for (int k = 0; k < 12; k++) ay[k] = acc[k] - ay[k];
    SpinorIO<P>::store(y2, rhs_ptr_w<P>(a.out, s.l, s.rhs, stride), rhs_norm(a.out, s.l, s.rhs, stride), stride, i);
    SpinorIO<P>::store(ay, rhs_ptr_w<P>(a.out2, s.l, s.rhs, stride), rhs_norm(a.out2, s.l, s.rhs, stride), stride, i);
    return;
  }
  if (MODE & MODE_XPAY) {
    cpx<R> xv[12];
    SpinorIO<P>::load(xv, rhs_ptr<P>(a.x, s.l, s.rhs, stride), rhs_norm(a.x, s.l, s.rhs, stride), stride, i);
    const R beta = R(a.beta[s.l]);
    if (MODE & MODE_PRE) {
      cpx<R> cx[12];
      CloverIO<P>::apply(cx, xv, a.cpre[s.l], a.cpre_norm[s.l], stride, i);
#pragma unroll
      for (int k = 0; k < 12; k++) acc[k] = acc[k] + beta * cx[k];
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) acc[k] = acc[k] + beta * xv[k];
    }
    if (EPI == EPI_ALPHA) {
      cpx<R> fv[12];
      SpinorIO<P>::load(fv, rhs_ptr<P>(a.f, s.l, s.rhs, stride), rhs_norm(a.f, s.l, s.rhs, stride), stride, i);
      dot_acc(red, fv, acc);
    } else if (EPI == EPI_OMEGA) {
      dot_acc(red, acc, xv);
      red[2] += norm_site(acc);
    } else if (EPI == EPI_CGALPHA || EPI == EPI_CGZ) {
      red[0] += norm_site(acc);
    }
  }
  if (MODE & MODE_POST) {
    cpx<R> y2[12];
    CloverIO<P>::apply(y2, acc, a.cpost[s.l], a.cpost_norm[s.l], stride, i);
    SpinorIO<P>::store(y2, rhs_ptr_w<P>(a.out, s.l, s.rhs, stride), rhs_norm(a.out, s.l, s.rhs, stride), stride, i);
  } else {
    SpinorIO<P>::store(acc, rhs_ptr_w<P>(a.out, s.l, s.rhs, stride), rhs_norm(a.out, s.l, s.rhs, stride), stride, i);
  }
}

template <int P, bool DAG, int MODE, int EPI>
__global__ void __launch_bounds__(256) dslash_kernel(const __grid_constant__ DslashArgs a) {
  const Slice s = find_slice(a.b, blockIdx.x);
  if (a.active && !a.active[s.slot]) return;
  const LatGeom& g = a.b.lat[s.l];
  const long i = (long)s.chunk * blockDim.x + threadIdx.x;
  double red[3] = {0.0, 0.0, 0.0};
  if (i < g.vh) dslash_site<P, DAG, MODE, EPI>(a, s, g, i, red);
  if constexpr (EPI != EPI_NONE)
    slice_reduce<3>(red, s, g.nchunk, a.maxch, a.partials, a.counters, a.sc,
                    [](Scalars& c, const double* t) { epi_finalize<EPI>(c, t); });
}

// Clover-only: out = C x  (used for A_oo^-1 b_o and stand-alone clover applies).
struct CloverArgs {
  Batch b;
  FieldRef out, x;
  const void* c[MAXLAT];
  const float* c_norm[MAXLAT];
  const int* active;
};

template <int P>
__global__ void __launch_bounds__(256) clover_kernel(const __grid_constant__ CloverArgs a) {
  using R = typename Traits<P>::R;
  const Slice s = find_slice(a.b, blockIdx.x);
  if (a.active && !a.active[s.slot]) return;
  const LatGeom& g = a.b.lat[s.l];
  const long i = (long)s.chunk * blockDim.x + threadIdx.x;
  if (i >= g.vh) return;
  cpx<R> xv[12], y[12];
  SpinorIO<P>::load(xv, rhs_ptr<P>(a.x, s.l, s.rhs, g.stride), rhs_norm(a.x, s.l, s.rhs, g.stride), g.stride, i);
  CloverIO<P>::apply(y, xv, a.c[s.l], a.c_norm[s.l], g.stride, i);
  SpinorIO<P>::store(y, rhs_ptr_w<P>(a.out, s.l, s.rhs, g.stride), rhs_norm(a.out, s.l, s.rhs, g.stride), g.stride, i);
}

// ---------------------------------------------------------------------------
// Multi-RHS kernel: a CTA covers TS (8, 16 or 32) consecutive output sites and every
// right-hand side.  Links and clover of the tile are read from memory once,
// unpacked (12-real reconstruction, 16-bit scaling) into shared memory, and
// reused by all RHS, as are the neighbour indices; each thread then computes one
// (site, rhs) pair.  The TS threads of one RHS are consecutive lanes of a warp.  Fused reductions write one partial per (RHS,
// CTA) and are finalised by tc_epi_finalize_kernel.
constexpr int MR_SITES = 8;  // smallest tile (sizes the reduction partials)

// Unpack chunk k of the packed clover term of site i into reals r[0..n) (n per chunk:
// 2 for FP64, 4 for FP32, 8 for the 16-bit formats, which carry one scale per site).
template <int P>
struct CloverChunk;
template <>
struct CloverChunk<F64> {
  static constexpr int NCH = 36, PER = 2;
  __device__ static void load(double r[2], const void* base, const float*, long stride, long i, int k) {
    const double2 v = ldcs(static_cast<const double2*>(base) + k * stride + i);
    r[0] = v.x;
    r[1] = v.y;
  }
};
template <>
struct CloverChunk<F32> {
  static constexpr int NCH = 18, PER = 4;
  __device__ static void load(float r[4], const void* base, const float*, long stride, long i, int k) {
    const float4 v = ldcs(static_cast<const float4*>(base) + k * stride + i);
    r[0] = v.x;
    r[1] = v.y;
    r[2] = v.z;
    r[3] = v.w;
  }
};
template <int P>
struct CloverChunk16 {
  static constexpr int NCH = 9, PER = 8;
  __device__ static void load(float r[8], const void* base, const float* norm, long stride, long i, int k) {
    const uint4 q = ldcs(static_cast<const uint4*>(base) + k * stride + i);
    const float n = ldcs(norm + i);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const float2 f = unpack2<P>(w[j]);
      r[2 * j] = f.x * n;
      r[2 * j + 1] = f.y * n;
    }
  }
};
template <>
struct CloverChunk<F16> : CloverChunk16<F16> {};
template <>
struct CloverChunk<BF16> : CloverChunk16<BF16> {};

// Per-site rows of reals in shared memory, read with 16-byte loads.  The row
// length is padded so that eight consecutive sites' 16-byte reads fall in
// distinct banks (row length in 4-byte words = 4 x odd, mod 32).
template <typename R>
struct SmemRow;
template <>
struct SmemRow<float> {
  static constexpr int LINK = 20, CLOV = 76, PER = 4;
  __device__ static void get(float* o, const float* row, int k) {
    const float4 v = reinterpret_cast<const float4*>(row)[k];
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
};
template <>
struct SmemRow<double> {
  static constexpr int LINK = 18, CLOV = 74, PER = 2;
  __device__ static void get(double* o, const double* row, int k) {
    const double2 v = reinterpret_cast<const double2*>(row)[k];
    o[0] = v.x;
    o[1] = v.y;
  }
};

// lower-triangle packing of a 6x6 block: entry k = r (r - 1) / 2 + c, c < r
__host__ __device__ constexpr int tri_row(int k) { return k < 1 ? 1 : k < 3 ? 2 : k < 6 ? 3 : k < 10 ? 4 : 5; }
__host__ __device__ constexpr int tri_col(int k) { return k - tri_row(k) * (tri_row(k) - 1) / 2; }

// y = C x for one Hermitian 6x6 block streamed from its shared-memory row (6 diagonal
// reals, then the 15 lower entries): each 16-byte read is consumed at once, in the
// same order of operations as hermitian6_apply
template <typename R>
__device__ __forceinline__ void hermitian6_apply_row(cpx<R> y[6], const R* row, const cpx<R> x[6]) {
  constexpr int PER = SmemRow<R>::PER;
#pragma unroll
  for (int q = 0; q < 36 / PER; q++) {
    R v[PER];
    SmemRow<R>::get(v, row, q);
#pragma unroll
    for (int j = 0; j < PER; j++) {
      const int e = q * PER + j;
      if (e < 6) {
        y[e] = v[j] * x[e];
      } else if ((e - 6) % 2 == 0) {
        const int k = (e - 6) / 2, r = tri_row(k), c = tri_col(k);
        const cpx<R> l = {v[j], v[j + 1]};
        cfma(y[r], l, x[c]);       // lower entry (r, c)
        cfma_conj(y[c], l, x[r]);  // upper entry (c, r) = conj(l)
      }
    }
  }
}

// y += beta C x for one block, streamed like hermitian6_apply_row (beta folded into
// each entry, so no separate C x is held)
template <typename R>
__device__ __forceinline__ void hermitian6_axpy_row(cpx<R> y[6], R beta, const R* row, const cpx<R> x[6]) {
  constexpr int PER = SmemRow<R>::PER;
#pragma unroll
  for (int q = 0; q < 36 / PER; q++) {
    R v[PER];
    SmemRow<R>::get(v, row, q);
#pragma unroll
    for (int j = 0; j < PER; j++) {
      const int e = q * PER + j;
      if (e < 6) {
        const R bd = beta * v[j];
        y[e].re = fma(bd, x[e].re, y[e].re);
        y[e].im = fma(bd, x[e].im, y[e].im);
      } else if ((e - 6) % 2 == 0) {
        const int k = (e - 6) / 2, r = tri_row(k), c = tri_col(k);
        const cpx<R> l = {beta * v[j], beta * v[j + 1]};
        cfma(y[r], l, x[c]);
        cfma_conj(y[c], l, x[r]);
      }
    }
  }
}

template <typename R>
__device__ __forceinline__ void clover_apply_smem(cpx<R> y[12], const cpx<R> x[12], const R* row) {
  hermitian6_apply_row(y, row, x);
  hermitian6_apply_row(y + 6, row + 36, x + 6);
}

// o = sign U h (ADJ: sign U^+ h) for both spin halves of h, U streamed from its
// shared-memory row (18 reals, row-major), in the order of link_mul
template <bool ADJ, typename R>
__device__ __forceinline__ void link_mul_row(const R* row, const cpx<R> h[6], cpx<R> o[6], R sign) {
  constexpr int PER = SmemRow<R>::PER;
#pragma unroll
  for (int k = 0; k < 6; k++) o[k] = {R(0), R(0)};
#pragma unroll
  for (int q = 0; q < (18 + PER - 1) / PER; q++) {
    R v[PER];
    SmemRow<R>::get(v, row, q);
#pragma unroll
    for (int j = 0; j < PER; j += 2) {
      const int e = (q * PER + j) / 2;
      if (e < 9) {
        const int a = e / 3, b = e % 3;
        const cpx<R> u = {v[j], v[j + 1]};
#pragma unroll
        for (int k = 0; k < 2; k++) {
          if (ADJ)
            cfma_conj(o[3 * k + b], u, h[3 * k + a]);  // (U^+)_{ba} = conj(U_ab)
          else
            cfma(o[3 * k + a], u, h[3 * k + b]);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 6; k++) o[k] = sign * o[k];
}

// A gathered neighbour spinor as it arrives from memory.  The 16-bit formats keep their
// packed halves and the site's norm; they are unpacked only when the hop is computed,
// and the norm is applied to the hop's link-multiply output (12 reals) instead of to
// the spinor (24 reals): the projection and the link multiply are linear.
template <int P>
struct RawSpinor {  // FP32: six 16-byte chunks
  float4 c[6];
};
template <>
struct RawSpinor<F64> {
  double2 c[12];
};
struct RawSpinor16 {
  uint4 c[3];
  float n;
};
template <>
struct RawSpinor<F16> : RawSpinor16 {};
template <>
struct RawSpinor<BF16> : RawSpinor16 {};

template <int P>
__device__ __forceinline__ void load_raw(RawSpinor<P>& r, const void* base, const float* norm, long stride, long j) {
  if constexpr (P == F64) {
    const double2* q = static_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) r.c[k] = ldg(q + k * stride + j);
  } else if constexpr (P == F32) {
    const float4* q = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++) r.c[k] = ldg(q + k * stride + j);
  } else {
    const uint4* q = static_cast<const uint4*>(base);
#pragma unroll
    for (int k = 0; k < 3; k++) r.c[k] = ldg(q + k * stride + j);
    r.n = ldg(norm + j);
  }
}

// unpack without the norm; returns the factor still to be applied (1, or the norm)
template <int P>
__device__ __forceinline__ typename Traits<P>::R unpack_raw(const RawSpinor<P>& r, cpx<typename Traits<P>::R> v[12]) {
  if constexpr (P == F64) {
#pragma unroll
    for (int k = 0; k < 12; k++) v[k] = {r.c[k].x, r.c[k].y};
    return 1.0;
  } else if constexpr (P == F32) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      v[2 * k] = {r.c[k].x, r.c[k].y};
      v[2 * k + 1] = {r.c[k].z, r.c[k].w};
    }
    return 1.f;
  } else {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint32_t w[4] = {r.c[k].x, r.c[k].y, r.c[k].z, r.c[k].w};
#pragma unroll
      for (int m = 0; m < 4; m++) {
        const float2 f = unpack2<P>(w[m]);
        v[4 * k + m] = {f.x, f.y};
      }
    }
    return r.n;
  }
}

// U_f, U_b: shared-memory rows of the forward link at the site and the backward
// link at the neighbour (18 reals each)
template <int P, int MU, bool DAG>
__device__ __forceinline__ void hop_dir_smem(cpx<typename Traits<P>::R> acc[12], const void* in, const float* in_norm,
                                             long stride, long jf, long jb, const typename Traits<P>::R* U_f,
                                             const typename Traits<P>::R* U_b, typename Traits<P>::R sf,
                                             typename Traits<P>::R sb) {
  using R = typename Traits<P>::R;
  constexpr int SF = DAG ? +1 : -1;
  constexpr int SB = -SF;
  cpx<R> psi[12], h[6], uh[6];
  RawSpinor<P> raw;
  load_raw<P>(raw, in, in_norm, stride, jf);
  R nf = unpack_raw<P>(raw, psi);
  project<MU, SF>(psi, h);
  link_mul_row<false>(U_f, h, uh, sf * nf);
  reconstruct_acc<MU, SF>(acc, uh);
  load_raw<P>(raw, in, in_norm, stride, jb);
  nf = unpack_raw<P>(raw, psi);
  project<MU, SB>(psi, h);
  link_mul_row<true>(U_b, h, uh, sb * nf);
  reconstruct_acc<MU, SB>(acc, uh);
}

struct SiteNbr {
  long jf[4], jb[4];
  int t;
};
__device__ __forceinline__ SiteNbr site_neighbours(const LatGeom& g, int p, long i) {
  SiteNbr n;
  const int lxh = g.lxh, Lx = g.dims[0], Ly = g.dims[1], Lz = g.dims[2], Lt = g.dims[3];
  const int xh = (int)(i % lxh);
  int rem = (int)(i / lxh);
  const int y = rem % Ly;
  rem /= Ly;
  const int z = rem % Lz;
  const int t = rem / Lz;
  const int x = 2 * xh + ((p + y + z + t) & 1);
  const long row = i - xh;
  const long plane = (long)lxh * Ly, vol3 = plane * Lz;
  n.jf[0] = row + ((x + 1 == Lx ? 0 : x + 1) >> 1);
  n.jb[0] = row + ((x == 0 ? Lx - 1 : x - 1) >> 1);
  n.jf[1] = (y + 1 == Ly) ? i - (long)(Ly - 1) * lxh : i + lxh;
  n.jb[1] = (y == 0) ? i + (long)(Ly - 1) * lxh : i - lxh;
  n.jf[2] = (z + 1 == Lz) ? i - (long)(Lz - 1) * plane : i + plane;
  n.jb[2] = (z == 0) ? i + (long)(Lz - 1) * plane : i - plane;
  n.jf[3] = (t + 1 == Lt) ? i - (long)(Lt - 1) * vol3 : i + vol3;
  n.jb[3] = (t == 0) ? i + (long)(Lt - 1) * vol3 : i - vol3;
  n.t = t;
  return n;
}

// ---------------------------------------------------------------------------
// Asynchronous staging of neighbour spinors (cp.async, 16-byte copies global ->
// shared memory that do not occupy registers while in flight).  A thread's slot of
// a stage holds the CH chunks of one spinor at [chunk][thread] (16 bytes each) and,
// for the 16-bit formats, its norm.
template <int P>
struct SpinorStage;
template <>
struct SpinorStage<F64> {
  static constexpr int CH = 12;
  static constexpr bool NORM = false;
};
template <>
struct SpinorStage<F32> {
  static constexpr int CH = 6;
  static constexpr bool NORM = false;
};
template <int P>
struct SpinorStage16 {
  static constexpr int CH = 3;
  static constexpr bool NORM = true;
};
template <>
struct SpinorStage<F16> : SpinorStage16<F16> {};
template <>
struct SpinorStage<BF16> : SpinorStage16<BF16> {};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// the "memory" clobbers keep the compiler from moving shared-memory reads of a
// slot past the copies that refill it, or before the wait that completes it
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// issue the copies of the spinor at site j into stage slot (chunk stride nt uint4)
template <int P>
__device__ __forceinline__ void stage_issue(uint4* slot, float* nslot, int nt, const void* base, const float* norm,
                                            long stride, long j) {
  const uint4* g = static_cast<const uint4*>(base);
#pragma unroll
  for (int k = 0; k < SpinorStage<P>::CH; k++) cp_async16(slot + k * nt, g + k * stride + j);
  if (SpinorStage<P>::NORM) cp_async4(nslot, norm + j);
}

template <int P>
__device__ __forceinline__ void stage_read(cpx<float> v[12], const uint4* slot, const float* nslot, int nt);
__device__ __forceinline__ void stage_read_f64(cpx<double> v[12], const uint4* slot, int nt) {
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const double2 d = reinterpret_cast<const double2*>(slot)[k * nt];
    v[k] = {d.x, d.y};
  }
}
template <>
__device__ __forceinline__ void stage_read<F32>(cpx<float> v[12], const uint4* slot, const float*, int nt) {
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const float4 f = reinterpret_cast<const float4*>(slot)[k * nt];
    v[2 * k] = {f.x, f.y};
    v[2 * k + 1] = {f.z, f.w};
  }
}
template <int P>
__device__ __forceinline__ void stage_read16(cpx<float> v[12], const uint4* slot, const float* nslot, int nt) {
  const float n = *nslot;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const uint4 q = slot[k * nt];
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int m = 0; m < 4; m++) {
      const float2 f = unpack2<P>(w[m]);
      v[4 * k + m] = {f.x * n, f.y * n};
    }
  }
}
template <>
__device__ __forceinline__ void stage_read<F16>(cpx<float> v[12], const uint4* slot, const float* nslot, int nt) {
  stage_read16<F16>(v, slot, nslot, nt);
}
template <>
__device__ __forceinline__ void stage_read<BF16>(cpx<float> v[12], const uint4* slot, const float* nslot, int nt) {
  stage_read16<BF16>(v, slot, nslot, nt);
}

// one hop (direction h = 2 mu + backward) from an already loaded neighbour spinor
template <int MU, bool BACK, bool DAG, typename R>
__device__ __forceinline__ void hop_from(cpx<R> acc[12], const cpx<R> psi[12], const R* U, R sign) {
  constexpr int SF = DAG ? +1 : -1;
  constexpr int S = BACK ? -SF : SF;
  cpx<R> h[6], uh[6];
  project<MU, S>(psi, h);
  link_mul_row<BACK>(U, h, uh, sign);
  reconstruct_acc<MU, S>(acc, uh);
}

// Register cap: every tile size keeps 64 registers per thread (five 192-thread or ten
// 96-thread CTAs per SM for 12 RHS).  A 32-site CTA covers MR32_RPC right-hand sides
// (the RHS of a tile are split over gridDim.y CTAs), so that each warp is 32 sites of
// one RHS: a 16-byte shared-memory read of the staged links then returns 32 distinct
// values in its four wavefronts, where a warp of 16 sites x 2 RHS reads every value
// twice.  Each of the tile's CTAs stages the tile's links and clover (L2 hits after
// the first).
constexpr int MR32_RPC = 6;
template <int TS>
struct MrhsBounds;
template <>
struct MrhsBounds<8> {
  static constexpr int THREADS = 128, MIN_BLOCKS = 8;
};
template <>
struct MrhsBounds<16> {
  static constexpr int THREADS = 256, MIN_BLOCKS = 4;
};
template <>
struct MrhsBounds<32> {
  static constexpr int THREADS = 32 * MR32_RPC, MIN_BLOCKS = 5;
};

// ASYNC: the eight neighbour spinors of a thread are staged through shared memory
// with cp.async, two hops in flight (dynamic shared memory: 2 stages x CH chunks x
// blockDim 16-byte slots, plus norms)
// PF: the neighbour spinor of the next hop is loaded into registers, as it arrives
// from memory (packed for the 16-bit formats), before the current hop is computed
// (software pipelining: one hop's gathers always in flight); FP32 and FP64 with the
// register cap of the staged variant, the 16-bit formats (13 registers in flight) with
// that of the plain kernel
template <int P, bool DAG, int MODE, int EPI, int TS, bool ASYNC = false, bool PF = false>
__global__ void __launch_bounds__(MrhsBounds<TS>::THREADS,
                                  (P == F64 ? 1 : (ASYNC || (PF && P == F32)) ? MrhsBounds<TS>::MIN_BLOCKS - 1
                                                                               : MrhsBounds<TS>::MIN_BLOCKS))
    dslash_mrhs_kernel(const __grid_constant__ DslashArgs a) {
  using R = typename Traits<P>::R;
  constexpr bool CLOV = (MODE & MODE_POST) || (MODE & MODE_PRE);
  constexpr int LROW = SmemRow<R>::LINK, CROW = SmemRow<R>::CLOV;
  __shared__ __align__(16) R Us[8][TS][LROW];  // links: 2 mu (fwd at the site), 2 mu + 1 (bwd at the neighbour)
  __shared__ __align__(16) R Cs[CLOV ? TS : 1][CLOV ? CROW : 4];  // unpacked clover, 72 reals per site
  __shared__ int Nb[8][TS];               // neighbour indices within the other parity: 2 mu fwd, 2 mu + 1 bwd
  __shared__ unsigned char Tb[TS];        // bit 0: forward t hop wraps, bit 1: backward t hop wraps
  const Slice s = find_slice(a.b, blockIdx.x);  // one slice per lattice
  const LatGeom& g = a.b.lat[s.l];
  const int nrhs = a.nrhs_tc;
  const int slot0 = s.l * nrhs;
  const int p = a.out_parity;
  const long stride = g.stride;
  long tile = s.chunk;
  if (g.zblk > 0) {
    // blocked order (z blocks outermost, then t, z in the block, y, x tile): the t
    // neighbours of a site are gathered Ly * zblk tiles apart instead of Ly * Lz, so
    // they are still in L2 (tiles are whole x rows or exact parts of one)
    const int tpr = g.lxh / TS, Ly = g.dims[1], Lz = g.dims[2], Lt = g.dims[3], bz = g.zblk;
    long q = tile;
    const int xt = (int)(q % tpr);
    q /= tpr;
    const int y = (int)(q % Ly);
    q /= Ly;
    const int zz = (int)(q % bz);
    q /= bz;
    const int t = (int)(q % Lt);
    const int zb = (int)(q / Lt);
    tile = (((long)t * Lz + zb * bz + zz) * Ly + y) * tpr + xt;
  }
  const long site0 = tile * TS;

  // phase 0: coordinates and neighbours of the tile's sites, once for all RHS
  if (threadIdx.x < TS) {
    const long i = site0 + threadIdx.x;
    if (i < g.vh) {
      const SiteNbr n = site_neighbours(g, p, i);
#pragma unroll
      for (int mu = 0; mu < 4; mu++) {
        Nb[2 * mu][threadIdx.x] = (int)n.jf[mu];
        Nb[2 * mu + 1][threadIdx.x] = (int)n.jb[mu];
      }
      Tb[threadIdx.x] = (n.t + 1 == g.dims[3] ? 1 : 0) | (n.t == 0 ? 2 : 0);
    }
  }
  __syncthreads();
  // phase 1: links and clover of the tile, unpacked to R.  Factors that are the
  // same for every RHS are applied here, once per site instead of once per (site,
  // RHS): the t-hop weights (boundary sign, anisotropy) go into the t links, and
  // alpha goes into the links (XPAY) or into the clover term applied after the hops
  // (POST); beta goes into the clover term applied to x (XPAY with PRE).
  const R alpha = R(a.alpha[s.l]);
  const R beta = R(a.beta[s.l]);
  constexpr bool ALPHA_IN_LINKS = !(MODE & MODE_POST);
  for (int e = threadIdx.x; e < 8 * TS; e += blockDim.x) {
    const int ls = e % TS, d = e / TS, mu = d >> 1;
    const long i = site0 + ls;
    cpx<R> u[3][3];
    if (i < g.vh) {
      // each link is read once per launch: evict-first, leaving L2 to the gathered spinors
      if (d & 1)
        LinkIO<P>::template load<true>(u, a.gauge[s.l][1 - p], stride, Nb[d][ls], mu);
      else
        LinkIO<P>::template load<true>(u, a.gauge[s.l][p], stride, i, mu);
    } else {
#pragma unroll
      for (int k = 0; k < 9; k++) u[k / 3][k % 3] = {R(0), R(0)};
    }
    R f = ALPHA_IN_LINKS ? alpha : R(1);
    if (d >= 6) f = f * hop_t_weight<R>(g, (Tb[ls] & (d == 6 ? 1 : 2)) != 0);
#pragma unroll
    for (int k = 0; k < 9; k++) {
      Us[d][ls][2 * k] = f * u[k / 3][k % 3].re;
      Us[d][ls][2 * k + 1] = f * u[k / 3][k % 3].im;
    }
  }
  if (CLOV) {
    using CC = CloverChunk<P>;
    const void* cb = (MODE & MODE_POST) ? a.cpost[s.l] : a.cpre[s.l];
    const float* cn = (MODE & MODE_POST) ? a.cpost_norm[s.l] : a.cpre_norm[s.l];
    const R cf = (MODE & MODE_POST) ? alpha : beta;
    for (int e = threadIdx.x; e < CC::NCH * TS; e += blockDim.x) {
      const int ls = e % TS, k = e / TS;
      const long i = site0 + ls;
      R r[CC::PER];
      if (i < g.vh) {
        CC::load(r, cb, cn, stride, i, k);
      } else {
#pragma unroll
        for (int j = 0; j < CC::PER; j++) r[j] = R(0);
      }
#pragma unroll
      for (int j = 0; j < CC::PER; j++) Cs[CLOV ? ls : 0][CLOV ? CC::PER * k + j : 0] = cf * r[j];
    }
  }
  __syncthreads();

  // phase 2: thread = (site ls, rhs); the TS threads of one rhs are consecutive lanes
  // (blockIdx.y > 0 only for 32-site tiles, whose RHS are split over CTAs)
  const int ls = threadIdx.x % TS, rhs = (int)blockIdx.y * (int)(blockDim.x / TS) + (int)(threadIdx.x / TS);
  const long i = site0 + ls;
  double red[3] = {0.0, 0.0, 0.0};
  const bool valid = rhs < nrhs && i < g.vh && (!a.active || a.active[slot0 + rhs]);
  if (valid) {
    const void* in = rhs_ptr<P>(a.in, s.l, rhs, stride);
    const float* in_norm = rhs_norm(a.in, s.l, rhs, stride);
    cpx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = {R(0), R(0)};
    // the t-hop weights are in the staged t links
    const R sf = R(1), sb = R(1);
    if constexpr (ASYNC) {
      extern __shared__ uint4 stage_mem[];
      const int nt = blockDim.x;
      constexpr int CH = SpinorStage<P>::CH;
      uint4* slot[2] = {stage_mem + threadIdx.x, stage_mem + CH * nt + threadIdx.x};
      float* nslot[2] = {reinterpret_cast<float*>(stage_mem + 2 * CH * nt) + threadIdx.x,
                         reinterpret_cast<float*>(stage_mem + 2 * CH * nt) + nt + threadIdx.x};
      stage_issue<P>(slot[0], nslot[0], nt, in, in_norm, stride, Nb[0][ls]);
      cp_async_commit();
      stage_issue<P>(slot[1], nslot[1], nt, in, in_norm, stride, Nb[1][ls]);
      cp_async_commit();
#pragma unroll
      for (int hh = 0; hh < 8; hh++) {
        if (hh < 7)
          cp_async_wait<1>();
        else
          cp_async_wait<0>();
        cpx<R> psi[12];
        if constexpr (P == F64)
          stage_read_f64(psi, slot[hh & 1], nt);
        else
          stage_read<P>(psi, slot[hh & 1], nslot[hh & 1], nt);
        const R sign = hh == 6 ? sf : hh == 7 ? sb : R(1);
        switch (hh) {
          case 0: hop_from<0, false, DAG>(acc, psi, Us[0][ls], sign); break;
          case 1: hop_from<0, true, DAG>(acc, psi, Us[1][ls], sign); break;
          case 2: hop_from<1, false, DAG>(acc, psi, Us[2][ls], sign); break;
          case 3: hop_from<1, true, DAG>(acc, psi, Us[3][ls], sign); break;
          case 4: hop_from<2, false, DAG>(acc, psi, Us[4][ls], sign); break;
          case 5: hop_from<2, true, DAG>(acc, psi, Us[5][ls], sign); break;
          case 6: hop_from<3, false, DAG>(acc, psi, Us[6][ls], sign); break;
          default: hop_from<3, true, DAG>(acc, psi, Us[7][ls], sign); break;
        }
        // the slot's values are consumed: refill it with hop hh + 2
        if (hh + 2 < 8) {
          stage_issue<P>(slot[hh & 1], nslot[hh & 1], nt, in, in_norm, stride, Nb[hh + 2][ls]);
          cp_async_commit();
        }
      }
    } else if constexpr (PF) {
      RawSpinor<P> nxt;
      load_raw<P>(nxt, in, in_norm, stride, Nb[0][ls]);
#pragma unroll
      for (int hh = 0; hh < 8; hh++) {
        const RawSpinor<P> cur = nxt;
        if (hh < 7) load_raw<P>(nxt, in, in_norm, stride, Nb[hh + 1][ls]);
        cpx<R> psi[12];
        const R sc = unpack_raw<P>(cur, psi);
        const R sign = (hh == 6 ? sf : hh == 7 ? sb : R(1)) * sc;
        switch (hh) {
          case 0: hop_from<0, false, DAG>(acc, psi, Us[0][ls], sign); break;
          case 1: hop_from<0, true, DAG>(acc, psi, Us[1][ls], sign); break;
          case 2: hop_from<1, false, DAG>(acc, psi, Us[2][ls], sign); break;
          case 3: hop_from<1, true, DAG>(acc, psi, Us[3][ls], sign); break;
          case 4: hop_from<2, false, DAG>(acc, psi, Us[4][ls], sign); break;
          case 5: hop_from<2, true, DAG>(acc, psi, Us[5][ls], sign); break;
          case 6: hop_from<3, false, DAG>(acc, psi, Us[6][ls], sign); break;
          default: hop_from<3, true, DAG>(acc, psi, Us[7][ls], sign); break;
        }
      }
    } else {
      hop_dir_smem<P, 0, DAG>(acc, in, in_norm, stride, Nb[0][ls], Nb[1][ls], Us[0][ls], Us[1][ls], R(1), R(1));
      hop_dir_smem<P, 1, DAG>(acc, in, in_norm, stride, Nb[2][ls], Nb[3][ls], Us[2][ls], Us[3][ls], R(1), R(1));
      hop_dir_smem<P, 2, DAG>(acc, in, in_norm, stride, Nb[4][ls], Nb[5][ls], Us[4][ls], Us[5][ls], R(1), R(1));
      hop_dir_smem<P, 3, DAG>(acc, in, in_norm, stride, Nb[6][ls], Nb[7][ls], Us[6][ls], Us[7][ls], sf, sb);
    }
    // alpha is in the staged links, or (POST) in the staged clover term
    if (MODE & MODE_XPAY) {
      cpx<R> xv[12];
      SpinorIO<P>::load_cs(xv, rhs_ptr<P>(a.x, s.l, rhs, stride), rhs_norm(a.x, s.l, rhs, stride), stride, i);
      if (MODE & MODE_PRE) {
        // beta is in the staged clover term
        hermitian6_axpy_row(acc, R(1), Cs[CLOV ? ls : 0], xv);
        hermitian6_axpy_row(acc + 6, R(1), Cs[CLOV ? ls : 0] + 36, xv + 6);
      } else {
#pragma unroll
        for (int k = 0; k < 12; k++) acc[k] = acc[k] + beta * xv[k];
      }
      if (EPI == EPI_ALPHA) {
        cpx<R> fv[12];
        SpinorIO<P>::load_cs(fv, rhs_ptr<P>(a.f, s.l, rhs, stride), rhs_norm(a.f, s.l, rhs, stride), stride, i);
        dot_acc(red, fv, acc);
      } else if (EPI == EPI_OMEGA) {
        dot_acc(red, acc, xv);
        red[2] += norm_site(acc);
      } else if (EPI == EPI_CGALPHA || EPI == EPI_CGZ) {
        red[0] += norm_site(acc);
      }
    }
    if (MODE & MODE_POST) {
      cpx<R> y2[12];
      clover_apply_smem<R>(y2, acc, Cs[CLOV ? ls : 0]);
      SpinorIO<P>::template store<true>(y2, rhs_ptr_w<P>(a.out, s.l, rhs, stride), rhs_norm(a.out, s.l, rhs, stride),
                                        stride, i);
    } else {
      SpinorIO<P>::template store<true>(acc, rhs_ptr_w<P>(a.out, s.l, rhs, stride), rhs_norm(a.out, s.l, rhs, stride),
                                        stride, i);
    }
  }
  if constexpr (EPI != EPI_NONE) {
    // the block size is a multiple of 32, so every lane of the warp takes part
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
      for (int o = TS / 2; o; o >>= 1) red[k] += __shfl_xor_sync(0xffffffffu, red[k], o);
    if (ls == 0 && rhs < nrhs) {
      double* dst = a.partials + ((size_t)(slot0 + rhs) * a.maxch + s.chunk) * 3;
      dst[0] = red[0];
      dst[1] = red[1];
      dst[2] = red[2];
    }
  }
}

// sums the per-CTA partials of every slot of a multi-RHS launch and runs the finaliser
struct TcChunks {
  int nch[MAXLAT];  // CTAs (partials) per lattice
  int nrhs;
};

// Two stages in one launch: block (b, slot) adds the partials of its contiguous
// range of CTAs in a fixed order and stores the sum in place of the range's first
// partial (which only this block reads); the last block of the slot to finish
// (atomic ticket) adds the EPI_FIN_BLOCKS range sums in index order and runs the
// finaliser.  The result does not depend on timing.  A single block per slot
// summing every partial (65,536 of them at 32^3x64) took about 70 us.
constexpr int EPI_FIN_BLOCKS = 64;

template <int EPI>
__global__ void __launch_bounds__(256) tc_epi_finalize_kernel(double* __restrict__ partials, int maxch, TcChunks ch,
                                                              const int* __restrict__ active,
                                                              unsigned* __restrict__ counters, Scalars* sc) {
  const int slot = blockIdx.y, b = blockIdx.x;
  if (active && !active[slot]) return;
  const int n = ch.nch[slot / ch.nrhs];
  const int per = (n + EPI_FIN_BLOCKS - 1) / EPI_FIN_BLOCKS;
  const int c_lo = b * per, c_hi = min(n, c_lo + per);
  double* part = partials + (size_t)slot * maxch * 3;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int c = c_lo + (int)threadIdx.x; c < c_hi; c += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 3; k++) acc[k] += __ldcg(part + (size_t)c * 3 + k);
  }
  __shared__ double sh[3][8];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sh[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (c_lo < c_hi) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        double v = 0.0;
        for (int w = 0; w < nw; w++) v += sh[k][w];
        part[(size_t)c_lo * 3 + k] = v;
      }
    }
    __threadfence();
    const unsigned ticket = atomicAdd(&counters[slot], 1u);
    last = (ticket == (unsigned)gridDim.x - 1u);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double tot[3] = {0.0, 0.0, 0.0};
  for (int bb = 0; bb < (int)gridDim.x; bb++) {
    const int c = bb * per;
    if (c >= n) break;
#pragma unroll
    for (int k = 0; k < 3; k++) tot[k] += __ldcg(part + (size_t)c * 3 + k);
  }
  epi_finalize<EPI>(sc[slot], tot);
  counters[slot] = 0u;
}

inline cudaError_t launch_epi_finalize(int epi, const DslashArgs& a, cudaStream_t st) {
  TcChunks ch;
  ch.nrhs = a.nrhs_tc;
  for (int l = 0; l < MAXLAT; l++) ch.nch[l] = l < a.b.nlat ? a.b.lat[l].nchunk : 0;
  const dim3 grid(EPI_FIN_BLOCKS, a.b.nlat * a.nrhs_tc);
  switch (epi) {
    case EPI_ALPHA: tc_epi_finalize_kernel<EPI_ALPHA><<<grid, 256, 0, st>>>(a.partials, a.maxch, ch, a.active, a.counters, a.sc); break;
    case EPI_OMEGA: tc_epi_finalize_kernel<EPI_OMEGA><<<grid, 256, 0, st>>>(a.partials, a.maxch, ch, a.active, a.counters, a.sc); break;
    case EPI_CGALPHA: tc_epi_finalize_kernel<EPI_CGALPHA><<<grid, 256, 0, st>>>(a.partials, a.maxch, ch, a.active, a.counters, a.sc); break;
    case EPI_CGZ: tc_epi_finalize_kernel<EPI_CGZ><<<grid, 256, 0, st>>>(a.partials, a.maxch, ch, a.active, a.counters, a.sc); break;
    default: return cudaSuccess;
  }
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_dslash_mrhs(const DslashArgs& a, bool dagger, int mode, int ts, cudaStream_t st,
                               bool async = false, bool pf = false);

// dynamic shared memory of the staged variant for `threads` threads
template <int P>
inline size_t mrhs_stage_bytes(int threads) {
  return (size_t)2 * SpinorStage<P>::CH * threads * 16 + (SpinorStage<P>::NORM ? (size_t)2 * threads * 4 : 0);
}

template <typename K>
inline cudaError_t allow_dynamic_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define WCL_MRHS_CASE(P, DAG, MODE, EPI)                                                         \
  case (MODE) | ((DAG) ? 16 : 0) | ((EPI) << 5):                                                \
    if (async) {                                                                                \
      const size_t sm = mrhs_stage_bytes<P>(threads);                                           \
      cudaError_t ea = allow_dynamic_smem(dslash_mrhs_kernel<P, DAG, MODE, EPI, 16, true>, sm); \
      if (ea != cudaSuccess) return ea;                                                         \
      dslash_mrhs_kernel<P, DAG, MODE, EPI, 16, true><<<a.b.total_blocks, threads, sm, st>>>(a); \
    } else if (pf)                                                                              \
      dslash_mrhs_kernel<P, DAG, MODE, EPI, 16, false, true><<<a.b.total_blocks, threads, 0, st>>>(a); \
    else if (ts == 32)                                                                          \
      dslash_mrhs_kernel<P, DAG, MODE, EPI, 32>                                                 \
          <<<dim3(a.b.total_blocks, (a.nrhs_tc + MR32_RPC - 1) / MR32_RPC), 32 * std::min(a.nrhs_tc, MR32_RPC), 0, st>>>(a); \
    else if (ts == 8)                                                                           \
      dslash_mrhs_kernel<P, DAG, MODE, EPI, 8><<<a.b.total_blocks, threads, 0, st>>>(a);        \
    else                                                                                        \
      dslash_mrhs_kernel<P, DAG, MODE, EPI, 16><<<a.b.total_blocks, threads, 0, st>>>(a);       \
    fin = EPI;                                                                                  \
    break;

// ts: sites per CTA (8, 16 or 32); the geometry a.b must have been built with that tile
#define WCL_DEFINE_MRHS_LAUNCHER(P)                                                              \
  template <>                                                                                    \
  cudaError_t launch_dslash_mrhs<P>(const DslashArgs& a, bool dagger, int mode, int ts, cudaStream_t st, bool async, \
                                    bool pf) {                                                   \
    if ((async || pf) && ts != 16) return cudaErrorInvalidValue;                                 \
    const int threads = (ts * a.nrhs_tc + 31) / 32 * 32;                                         \
    int fin = 0;                                                                                 \
    switch (mode | (dagger ? 16 : 0)) {                                                          \
      WCL_MRHS_CASE(P, false, MODE_POST, EPI_NONE)                                               \
      WCL_MRHS_CASE(P, true, MODE_POST, EPI_NONE)                                                \
      WCL_MRHS_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_NONE)                                    \
      WCL_MRHS_CASE(P, true, MODE_XPAY | MODE_PRE, EPI_NONE)                                     \
      WCL_MRHS_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_ALPHA)                                   \
      WCL_MRHS_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_OMEGA)                                   \
      WCL_MRHS_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_CGALPHA)                                 \
      WCL_MRHS_CASE(P, true, MODE_XPAY | MODE_PRE, EPI_CGZ)                                      \
      default: return cudaErrorInvalidValue;                                                     \
    }                                                                                            \
    cudaError_t e = cudaGetLastError();                                                          \
    if (e != cudaSuccess) return e;                                                              \
    return launch_epi_finalize(fin, a, st);                                                      \
  }

// host-side launchers (one instantiation set per precision translation unit)
template <int P>
cudaError_t launch_dslash(const DslashArgs& a, bool dagger, int mode, int block, cudaStream_t st);
template <int P>
cudaError_t launch_clover(const CloverArgs& a, int block, cudaStream_t st);

// the double-float operator only serves source preparation and residual replacement
#define WCL_DEFINE_DSLASH_LAUNCHERS_DF(P)                                                           \
  template <>                                                                                       \
  cudaError_t launch_dslash<P>(const DslashArgs& a, bool dagger, int mode, int block, cudaStream_t st) { \
    dim3 grid(a.b.total_blocks), blk(block);                                                        \
    switch (mode | (dagger ? 16 : 0)) {                                                             \
      WCL_DSLASH_CASE(P, false, MODE_POST, EPI_NONE)                                                \
      WCL_DSLASH_CASE(P, true, MODE_POST, EPI_NONE)                                                 \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_NONE)                                     \
      WCL_DSLASH_CASE(P, true, MODE_XPAY | MODE_PRE, EPI_NONE)                                      \
      WCL_DSLASH_CASE(P, false, MODE_XPAY, EPI_NONE)                                                \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_POST, EPI_NONE)                                    \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_POST | MODE_PRE | MODE_RECON, EPI_NONE)            \
      default: return cudaErrorInvalidValue;                                                        \
    }                                                                                               \
    return cudaGetLastError();                                                                      \
  }                                                                                                 \
  template <>                                                                                       \
  cudaError_t launch_clover<P>(const CloverArgs& a, int block, cudaStream_t st) {                   \
    clover_kernel<P><<<a.b.total_blocks, block, 0, st>>>(a);                                        \
    return cudaGetLastError();                                                                      \
  }

#define WCL_DSLASH_CASE(P, DAG, MODE, EPI)                                            \
  case (MODE) | ((DAG) ? 16 : 0) | ((EPI) << 5):                                       \
    dslash_kernel<P, DAG, MODE, EPI><<<grid, blk, 0, st>>>(a);                         \
    break;

#define WCL_DEFINE_DSLASH_LAUNCHERS(P)                                                              \
  template <>                                                                                       \
  cudaError_t launch_dslash<P>(const DslashArgs& a, bool dagger, int mode, int block, cudaStream_t st) { \
    dim3 grid(a.b.total_blocks), blk(block);                                                        \
    switch (mode | (dagger ? 16 : 0)) {                                                             \
      WCL_DSLASH_CASE(P, false, MODE_POST, EPI_NONE)                                                \
      WCL_DSLASH_CASE(P, true, MODE_POST, EPI_NONE)                                                 \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_NONE)                                     \
      WCL_DSLASH_CASE(P, true, MODE_XPAY | MODE_PRE, EPI_NONE)                                      \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_ALPHA)                                    \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_OMEGA)                                    \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_CGALPHA)                                  \
      WCL_DSLASH_CASE(P, true, MODE_XPAY | MODE_PRE, EPI_CGZ)                                       \
      WCL_DSLASH_CASE(P, false, MODE_XPAY, EPI_NONE)                                                \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_POST, EPI_NONE)                                    \
      WCL_DSLASH_CASE(P, false, MODE_XPAY | MODE_POST | MODE_PRE | MODE_RECON, EPI_NONE)            \
      default: return cudaErrorInvalidValue;                                                        \
    }                                                                                               \
    return cudaGetLastError();                                                                      \
  }                                                                                                 \
  template <>                                                                                       \
  cudaError_t launch_clover<P>(const CloverArgs& a, int block, cudaStream_t st) {                   \
    clover_kernel<P><<<a.b.total_blocks, block, 0, st>>>(a);                                        \
    return cudaGetLastError();                                                                      \
  }

}  // namespace wcl
