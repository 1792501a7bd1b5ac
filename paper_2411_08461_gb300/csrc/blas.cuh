// BLAS-1 updates and reductions over (lattice, rhs) slices, and the solver
// recurrences built from them.  Reductions accumulate in FP64: each thread sums
// its sites, warps combine with shuffles, blocks write one partial per slice,
// and the last block of a slice (atomic ticket) adds the partials in a fixed
// order -- so results are deterministic -- and runs the finalizer that derives
// the solver coefficients on the device.  No solver step needs the host.
#pragma once
#include "internal.cuh"

namespace wcl {

constexpr int RED_MAXCH = 512;  // blocks per slice for map / reduce kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

template <typename F>
__global__ void __launch_bounds__(256) map_kernel(const __grid_constant__ Batch b, const __grid_constant__ F f,
                                                  const int* __restrict__ active) {
  const Slice s = find_slice(b, blockIdx.x);
  if (active && !active[s.slot]) return;
  const LatGeom& g = b.lat[s.l];
  for (long i = (long)s.chunk * blockDim.x + threadIdx.x; i < g.vh; i += (long)g.nchunk * blockDim.x) f(s, g, i);
}

// Block-level reduction of NR doubles per thread for the slice s, one partial per
// block, and the finalizer run once per slice by its last block (atomic ticket;
// partials summed in a fixed order, so the result is deterministic).  Every
// thread of the block must call it.  fin(Scalars&, const double* tot).
template <int NR, typename Fin>
__device__ __forceinline__ void slice_reduce(double acc[NR], const Slice& s, int nchunk, int maxch,
                                             double* __restrict__ partials, unsigned* __restrict__ counters,
                                             Scalars* __restrict__ sc, const Fin& fin) {
  __shared__ double sh[NR][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NR; k++) {
    double v = warp_sum(acc[k]);
    if (lane == 0) sh[k][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NR; k++) {
      double v = lane < nw ? sh[k][lane] : 0.0;
      v = warp_sum(v);
      if (lane == 0) partials[((size_t)s.slot * maxch + s.chunk) * NR + k] = v;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(&counters[s.slot], 1u);
    last = (ticket == (unsigned)nchunk - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot[NR];
#pragma unroll
  for (int k = 0; k < NR; k++) tot[k] = 0.0;
  for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NR; k++) tot[k] += __ldcg(partials + ((size_t)s.slot * maxch + c) * NR + k);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NR; k++) {
    double v = warp_sum(tot[k]);
    if (lane == 0) sh[k][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NR; k++) {
      double v = lane < nw ? sh[k][lane] : 0.0;
      tot[k] = warp_sum(v);
    }
    if (lane == 0) {
      fin(sc[s.slot], tot);
      counters[s.slot] = 0u;
    }
  }
}

template <int NR, typename F>
__global__ void __launch_bounds__(256) reduce_kernel(const __grid_constant__ Batch b, const __grid_constant__ F f,
                                                     const int* __restrict__ active, double* __restrict__ partials,
                                                     unsigned* __restrict__ counters, Scalars* __restrict__ sc) {
  const Slice s = find_slice(b, blockIdx.x);
  if (active && !active[s.slot]) return;
  const LatGeom& g = b.lat[s.l];
  double acc[NR];
#pragma unroll
  for (int k = 0; k < NR; k++) acc[k] = 0.0;
  for (long i = (long)s.chunk * blockDim.x + threadIdx.x; i < g.vh; i += (long)g.nchunk * blockDim.x) f(s, g, i, acc);
  slice_reduce<NR>(acc, s, g.nchunk, RED_MAXCH, partials, counters, sc,
                   [&](Scalars& c, const double* t) { f.finalize(c, t); });
}

// ---------------------------------------------------------------------------
// field access shorthands inside functors
#define WCL_LD(P, NC, v, F)                                                                               \
  SpinorIO<P>::template load<NC>(v, rhs_ptr<P>(F, s.l, s.rhs, g.stride), rhs_norm(F, s.l, s.rhs, g.stride), \
                                 g.stride, i)
#define WCL_ST(P, v, F) \
  SpinorIO<P>::store(v, rhs_ptr_w<P>(F, s.l, s.rhs, g.stride), rhs_norm(F, s.l, s.rhs, g.stride), g.stride, i)

template <typename R>
__device__ __forceinline__ void dot_acc(double* acc, const cpx<R> a[12], const cpx<R> b[12]) {
  // acc[0] += Re <a,b>, acc[1] += Im <a,b>
  R re = 0, im = 0;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    re = fma(a[k].re, b[k].re, re);
    re = fma(a[k].im, b[k].im, re);
    im = fma(a[k].re, b[k].im, im);
    im = fma(-a[k].im, b[k].re, im);
  }
  acc[0] += (double)re;
  acc[1] += (double)im;
}
template <typename R>
__device__ __forceinline__ double norm_site(const cpx<R> a[12]) {
  R n = 0;
#pragma unroll
  for (int k = 0; k < 12; k++) n = fma(a[k].re, a[k].re, fma(a[k].im, a[k].im, n));
  return (double)n;
}
template <typename R>
__device__ __forceinline__ cpx<R> to_c(double2 z) {
  return {R(z.x), R(z.y)};
}

// ---------------------------------------------------------------------------
// generic helpers
template <int PO, int PI>
struct Convert {  // out = in
  FieldRef out, in;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    cpx<typename Traits<PI>::R> a[12];
    WCL_LD(PI, true, a, in);
    cpx<typename Traits<PO>::R> b[12];
#pragma unroll
    for (int k = 0; k < 12; k++) b[k] = {typename Traits<PO>::R(a[k].re), typename Traits<PO>::R(a[k].im)};
    WCL_ST(PO, b, out);
  }
};

template <int PX>
struct AddInto64 {  // x64 += xs; xs = 0
  FieldRef x64, xs;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    cpx<double> x[12];
    cpx<typename Traits<PX>::R> d[12];
    WCL_LD(F64, false, x, x64);
    WCL_LD(PX, false, d, xs);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      x[k] = x[k] + cpx<double>{double(d[k].re), double(d[k].im)};
      d[k] = {0, 0};
    }
    WCL_ST(F64, x, x64);
    WCL_ST(PX, d, xs);
  }
};

template <int PX>
struct AddInto64Split {  // x64 += xs; xs = 0; xdf = double-float copy of x64
  FieldRef x64, xs, xdf;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    cpx<double> x[12];
    cpx<typename Traits<PX>::R> d[12];
    WCL_LD(F64, false, x, x64);
    WCL_LD(PX, false, d, xs);
    cpx<dfloat> xd[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
      x[k] = x[k] + cpx<double>{double(d[k].re), double(d[k].im)};
      d[k] = {0, 0};
      xd[k] = {dfloat(x[k].re), dfloat(x[k].im)};
    }
    WCL_ST(F64, x, x64);
    WCL_ST(PX, d, xs);
    WCL_ST(DF64, xd, xdf);
  }
};

template <int P>
struct Norm2 {  // aux[k] (=|+=) ||a - b||^2  (b optional)
  FieldRef a, b;
  int k, accumulate, has_b;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    cpx<typename Traits<P>::R> x[12], y[12];
    WCL_LD(P, true, x, a);
    if (has_b) {
      WCL_LD(P, true, y, b);
#pragma unroll
      for (int c = 0; c < 12; c++) x[c] = x[c] - y[c];
    }
    acc[0] += norm_site(x);
  }
  __device__ void finalize(Scalars& c, const double* t) const { c.aux[k] = accumulate ? c.aux[k] + t[0] : t[0]; }
};

// ---------------------------------------------------------------------------
// BiCGStab (van der Vorst 1992) with device-side coefficients.
// Finalize modes for the rho reduction: NORMAL after an iteration, INIT at a
// (re)start (rho = alpha = omega = 1 before), REPLACE after a reliable update
// (the residual was replaced; beta is recomputed against the previous rho).
enum RhoMode { RHO_NORMAL = 0, RHO_INIT = 1, RHO_REPLACE = 2 };

__device__ __forceinline__ void bicg_rho_finalize(Scalars& c, double2 rho_new, double r2, int mode) {
  double2 prev;
  if (mode == RHO_INIT) {
    prev = make_double2(1, 0);
    c.alpha = make_double2(1, 0);
    c.omega = make_double2(1, 0);
    c.rho_prev = prev;
  } else if (mode == RHO_REPLACE) {
    prev = c.rho_prev;
  } else {
    prev = c.rho;
    c.rho_prev = prev;
  }
  if (cabs2(prev) == 0.0 || cabs2(c.omega) == 0.0 || !(r2 == r2)) {
    c.beta = make_double2(0, 0);
    c.flags |= 1;
  } else {
    c.beta = cmul(cdiv(rho_new, prev), cdiv(c.alpha, c.omega));
  }
  if (cabs2(rho_new) == 0.0 && r2 > 0.0) c.flags |= 1;
  c.rho = rho_new;
  c.r2 = r2;
}

template <int S>
struct BicgRho {  // rho' = <rhat, r>, r2 = ||r||^2
  FieldRef rhat, r;
  int mode;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    cpx<typename Traits<S>::R> a[12], b[12];
    WCL_LD(S, true, a, rhat);
    WCL_LD(S, true, b, r);
    dot_acc(acc, a, b);
    acc[2] += norm_site(b);
  }
  __device__ void finalize(Scalars& c, const double* t) const { bicg_rho_finalize(c, make_double2(t[0], t[1]), t[2], mode); }
};

template <int S>
struct BicgP {  // p = r + beta (p - omega v)
  FieldRef r, p, v;
  const Scalars* sc;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    using R = typename Traits<S>::R;
    const cpx<R> beta = to_c<R>(sc[s.slot].beta), omega = to_c<R>(sc[s.slot].omega);
    cpx<R> rr[12], pp[12], vv[12];
    WCL_LD(S, true, rr, r);
    WCL_LD(S, false, pp, p);
    WCL_LD(S, true, vv, v);
#pragma unroll
    for (int k = 0; k < 12; k++) pp[k] = rr[k] + beta * (pp[k] - omega * vv[k]);
    WCL_ST(S, pp, p);
  }
};

template <int S>
struct BicgAlpha {  // alpha = rho / <rhat, v>
  FieldRef rhat, v;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    cpx<typename Traits<S>::R> a[12], b[12];
    WCL_LD(S, true, a, rhat);
    WCL_LD(S, true, b, v);
    dot_acc(acc, a, b);
  }
  __device__ void finalize(Scalars& c, const double* t) const {
    const double2 rv = make_double2(t[0], t[1]);
    if (cabs2(rv) == 0.0 || !(t[0] == t[0])) {
      c.alpha = make_double2(0, 0);
      c.flags |= 1;
    } else {
      c.alpha = cdiv(c.rho, rv);
    }
  }
};

template <int S>
struct BicgS {  // s = r - alpha v  (in place in r)
  FieldRef r, v;
  const Scalars* sc;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    using R = typename Traits<S>::R;
    const cpx<R> alpha = to_c<R>(sc[s.slot].alpha);
    cpx<R> rr[12], vv[12];
    WCL_LD(S, false, rr, r);
    WCL_LD(S, true, vv, v);
#pragma unroll
    for (int k = 0; k < 12; k++) rr[k] = rr[k] - alpha * vv[k];
    WCL_ST(S, rr, r);
  }
};

template <int S>
struct BicgOmega {  // omega = <t, s> / <t, t>
  FieldRef t, sv;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    cpx<typename Traits<S>::R> a[12], b[12];
    WCL_LD(S, true, a, t);
    WCL_LD(S, true, b, sv);
    dot_acc(acc, a, b);
    acc[2] += norm_site(a);
  }
  __device__ void finalize(Scalars& c, const double* tt) const {
    if (!(tt[2] > 0.0)) {
      c.omega = make_double2(0, 0);
      c.flags |= 1;
    } else {
      c.omega = make_double2(tt[0] / tt[2], tt[1] / tt[2]);
    }
  }
};

template <int S, int X>
struct BicgUpdate {  // x += alpha p + omega s; r = s - omega t; then rho' and ||r||^2
  FieldRef xs, p, r, t, rhat;
  const Scalars* sc;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    using R = typename Traits<S>::R;
    using RX = typename Traits<X>::R;
    const double2 a2 = sc[s.slot].alpha, o2 = sc[s.slot].omega;
    cpx<R> pp[12], ss[12], tt[12], rh[12];
    cpx<RX> xx[12];
    // every load is issued before the first store: the stores go through pointers the
    // compiler cannot separate from rhat, so a later load would wait for them
    WCL_LD(S, true, pp, p);
    WCL_LD(S, false, ss, r);
    WCL_LD(S, true, tt, t);
    WCL_LD(X, false, xx, xs);
    WCL_LD(S, true, rh, rhat);
    const cpx<RX> ax = {RX(a2.x), RX(a2.y)}, ox = {RX(o2.x), RX(o2.y)};
    const cpx<R> om = to_c<R>(o2);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const cpx<RX> pk = {RX(pp[k].re), RX(pp[k].im)}, sk = {RX(ss[k].re), RX(ss[k].im)};
      xx[k] = xx[k] + ax * pk + ox * sk;
      ss[k] = ss[k] - om * tt[k];
    }
    WCL_ST(X, xx, xs);
    WCL_ST(S, ss, r);
    dot_acc(acc, rh, ss);
    acc[2] += norm_site(ss);
  }
  __device__ void finalize(Scalars& c, const double* t) const { bicg_rho_finalize(c, make_double2(t[0], t[1]), t[2], RHO_NORMAL); }
};

// One field of precision Q (F64 or DF64) read as FP64 values.
template <int Q>
__device__ __forceinline__ void load_as_f64(cpx<double> v[12], const void* base, long stride, long i);
template <>
__device__ __forceinline__ void load_as_f64<F64>(cpx<double> v[12], const void* base, long stride, long i) {
  SpinorIO<F64>::load<false>(v, base, nullptr, stride, i);
}
template <>
__device__ __forceinline__ void load_as_f64<DF64>(cpx<double> v[12], const void* base, long stride, long i) {
  cpx<dfloat> d[12];
  SpinorIO<DF64>::load<false>(d, base, nullptr, stride, i);
#pragma unroll
  for (int k = 0; k < 12; k++) v[k] = {double(d[k].re), double(d[k].im)};
}
template <>
__device__ __forceinline__ void load_as_f64<F32>(cpx<double> v[12], const void* base, long stride, long i) {
  cpx<float> d[12];
  SpinorIO<F32>::load<false>(d, base, nullptr, stride, i);
#pragma unroll
  for (int k = 0; k < 12; k++) v[k] = {double(d[k].re), double(d[k].im)};
}

// Reliable update: r64 holds y = A_ee x_e - kappa D_eo x_o in precision Q (x_o the
// reconstructed odd solution); r_e = b_e - y is formed in FP64 and equals the Schur
// residual b_hat - M_hat x_e; rS = r_e in the inner precision.  ro, when given, holds
// the odd residual b_o - (A_oo x_o - kappa D_oe x_e) of the reconstruction (precision
// Q).  aux[0] = ||r_e||^2, aux[3] = ||r_e||^2 + ||r_o||^2 = ||b - M x||^2 (the full true
// residual); BiCGStab also recomputes rho against rhat (REPLACE).  The sums of an IEEE
// FP64 update (Q = F64: every update that may end a solve) are FP64 throughout; those
// of a double-float update, which only decide whether an FP64 update follows, sum the
// residual as rounded to the inner precision per site (FP32 pipes; GB300's FP64 rate
// bounded this kernel) and add the per-site sums in FP64.  With Q = F32 (an early update of
// a 16-bit inner solve, made with the FP32 operator) r64 is an FP32 field.
template <int S, int Q>
struct ResidualReplace {
  FieldRef r64, bhat, rS, rhat, ro;
  int bicg;  // 1: BiCGStab rho REPLACE finalize; 0: CG (only the norm)
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    using R = typename Traits<S>::R;
    cpx<double> y[12], b[12];
    cpx<R> rh[12];
    if (bicg) WCL_LD(S, true, rh, rhat);
    if (ro.ptr[s.l]) {  // odd residual of the reconstruction (absent: x_o solves its rows exactly)
      load_as_f64<Q>(b, rhs_ptr<Q>(ro, s.l, s.rhs, g.stride), g.stride, i);
      acc[3] += norm_site(b);
    }
    load_as_f64<Q>(y, rhs_ptr<Q>(r64, s.l, s.rhs, g.stride), g.stride, i);
    WCL_LD(F64, true, b, bhat);
    cpx<R> rs[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
      y[k] = b[k] - y[k];
      rs[k] = {R(y[k].re), R(y[k].im)};
    }
    WCL_ST(S, rs, rS);
    if constexpr (Q == F64) {
      acc[0] += norm_site(y);
      if (bicg) {
        cpx<double> rhd[12];
#pragma unroll
        for (int k = 0; k < 12; k++) rhd[k] = {double(rh[k].re), double(rh[k].im)};
        double d[2] = {0, 0};
        dot_acc(d, rhd, y);
        acc[1] += d[0];
        acc[2] += d[1];
      }
    } else {
      acc[0] += norm_site(rs);
      if (bicg) {
        double d[2] = {0, 0};
        dot_acc(d, rh, rs);
        acc[1] += d[0];
        acc[2] += d[1];
      }
    }
  }
  __device__ void finalize(Scalars& c, const double* t) const {
    c.aux[0] = t[0];
    c.aux[3] = t[0] + t[3];
    if (bicg) {
      bicg_rho_finalize(c, make_double2(t[1], t[2]), t[0], RHO_REPLACE);
    } else {
      c.r2 = t[0];
    }
  }
};

// ---------------------------------------------------------------------------
// CG on the normal equations (CGNR), per iteration:
//   z = M^+ r; zz' = ||z||^2; beta = zz'/zz (0 on the first step); p = z + beta p
//   q = M p; alpha = zz' / ||q||^2; x += alpha p; r -= alpha q
// scalars: rho.x = zz, rho_prev.x = previous zz (0 before the first step)
template <int S>
struct CgZnorm {
  FieldRef z;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    cpx<typename Traits<S>::R> a[12];
    WCL_LD(S, true, a, z);
    acc[0] += norm_site(a);
  }
  __device__ void finalize(Scalars& c, const double* t) const {
    const double zz = t[0], prev = c.rho.x;
    c.beta = make_double2(prev > 0.0 ? zz / prev : 0.0, 0.0);
    c.rho_prev = c.rho;
    c.rho = make_double2(zz, 0.0);
    if (!(zz == zz)) c.flags |= 1;
  }
};

template <int S>
struct CgP {  // p = z + beta p
  FieldRef z, p;
  const Scalars* sc;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    using R = typename Traits<S>::R;
    const R beta = R(sc[s.slot].beta.x);
    cpx<R> zz[12], pp[12];
    WCL_LD(S, true, zz, z);
    WCL_LD(S, false, pp, p);
#pragma unroll
    for (int k = 0; k < 12; k++) pp[k] = zz[k] + beta * pp[k];
    WCL_ST(S, pp, p);
  }
};

template <int S>
struct CgAlpha {  // alpha = zz / ||q||^2
  FieldRef q;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    cpx<typename Traits<S>::R> a[12];
    WCL_LD(S, true, a, q);
    acc[0] += norm_site(a);
  }
  __device__ void finalize(Scalars& c, const double* t) const {
    if (!(t[0] > 0.0)) {
      c.alpha = make_double2(0, 0);
      c.flags |= 1;
    } else {
      c.alpha = make_double2(c.rho.x / t[0], 0.0);
    }
  }
};

template <int S, int X>
struct CgUpdate {  // x += alpha p; r -= alpha q; r2 = ||r||^2
  FieldRef xs, p, r, q;
  const Scalars* sc;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    using R = typename Traits<S>::R;
    using RX = typename Traits<X>::R;
    const double a = sc[s.slot].alpha.x;
    cpx<R> pp[12], rr[12], qq[12];
    cpx<RX> xx[12];
    WCL_LD(S, true, pp, p);
    WCL_LD(S, false, rr, r);
    WCL_LD(S, true, qq, q);
    WCL_LD(X, false, xx, xs);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      xx[k] = xx[k] + RX(a) * cpx<RX>{RX(pp[k].re), RX(pp[k].im)};
      rr[k] = rr[k] - R(a) * qq[k];
    }
    WCL_ST(X, xx, xs);
    WCL_ST(S, rr, r);
    acc[0] += norm_site(rr);
  }
  __device__ void finalize(Scalars& c, const double* t) const { c.r2 = t[0]; }
};

// ---------------------------------------------------------------------------
// host launch helpers
template <typename F>
cudaError_t run_map(const Batch& b, const F& f, const int* active, int block, cudaStream_t st) {
  map_kernel<F><<<b.total_blocks, block, 0, st>>>(b, f, active);
  return cudaGetLastError();
}
template <int NR, typename F>
cudaError_t run_reduce(const Batch& b, const F& f, const int* active, double* partials, unsigned* counters,
                       Scalars* sc, int block, cudaStream_t st) {
  reduce_kernel<NR, F><<<b.total_blocks, block, 0, st>>>(b, f, active, partials, counters, sc);
  return cudaGetLastError();
}

}  // namespace wcl

namespace wcl {

template <int S>
struct ZeroPair {  // a = b = 0
  FieldRef a, b;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    cpx<typename Traits<S>::R> z[12];
#pragma unroll
    for (int k = 0; k < 12; k++) z[k] = {0, 0};
    WCL_ST(S, z, a);
    WCL_ST(S, z, b);
  }
};

struct ResetCg {  // forget the CG search direction scale (beta = 0 on the next step)
  Scalars* sc;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    if (i == 0) {
      sc[s.slot].rho = make_double2(0, 0);
      sc[s.slot].beta = make_double2(0, 0);
    }
  }
};

}  // namespace wcl

namespace wcl {

// ---------------------------------------------------------------------------
// Flexible GCR helpers.  The Krylov sets Z, W hold m vectors of nrhs parity
// fields each: vector j of lattice l starts vstride[l] bytes after vector j-1.
constexpr int GCR_MAXK = 20;

template <int S>
__device__ __forceinline__ const void* kry_ptr(const FieldRef& base, const long* vstride, int j, int l, int rhs,
                                                long stride) {
  return static_cast<const char*>(rhs_ptr<S>(base, l, rhs, stride)) + (size_t)j * vstride[l];
}
template <int S>
__device__ __forceinline__ void* kry_ptr_w(const FieldRef& base, const long* vstride, int j, int l, int rhs,
                                           long stride) {
  return static_cast<char*>(rhs_ptr_w<S>(base, l, rhs, stride)) + (size_t)j * vstride[l];
}
__device__ __forceinline__ float* kry_norm(const FieldRef& base, const long* nvstride, int j, int l, int rhs,
                                           long stride) {
  return base.norm[l] ? base.norm[l] + (size_t)rhs * stride + (size_t)j * nvstride[l] : nullptr;
}

// beta_j = <W_j, w> for j < k; stored in betas[slot * GCR_MAXK + j]
template <int S>
struct GcrMultiDot {
  FieldRef W, w;
  long vstride[MAXLAT], nvstride[MAXLAT];
  int k;
  double2* betas;
  const Scalars* sc_base;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    cpx<typename Traits<S>::R> a[12], b[12];
    WCL_LD(S, true, b, w);
    for (int j = 0; j < k; j++) {
      SpinorIO<S>::load(a, kry_ptr<S>(W, vstride, j, s.l, s.rhs, g.stride), kry_norm(W, nvstride, j, s.l, s.rhs, g.stride),
                        g.stride, i);
      double d[2] = {0, 0};
      dot_acc(d, a, b);
      acc[2 * j] += d[0];
      acc[2 * j + 1] += d[1];
    }
  }
  __device__ void finalize(Scalars& c, const double* t) const {
    const long slot = &c - sc_base;
    for (int j = 0; j < k; j++) betas[slot * GCR_MAXK + j] = make_double2(t[2 * j], t[2 * j + 1]);
  }
};

// w -= sum_j beta_j W_j ; z -= sum_j beta_j Z_j
template <int S>
struct GcrMultiAxpy {
  FieldRef W, Z, w, z;
  long vstride[MAXLAT], nvstride[MAXLAT];
  int k;
  const double2* betas;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i) const {
    using R = typename Traits<S>::R;
    cpx<R> ww[12], zz[12], a[12];
    WCL_LD(S, false, ww, w);
    WCL_LD(S, false, zz, z);
    for (int j = 0; j < k; j++) {
      const double2 bj = betas[s.slot * GCR_MAXK + j];
      const cpx<R> b = {R(bj.x), R(bj.y)};
      SpinorIO<S>::load(a, kry_ptr<S>(W, vstride, j, s.l, s.rhs, g.stride), kry_norm(W, nvstride, j, s.l, s.rhs, g.stride),
                        g.stride, i);
#pragma unroll
      for (int c = 0; c < 12; c++) ww[c] = ww[c] - b * a[c];
      SpinorIO<S>::load(a, kry_ptr<S>(Z, vstride, j, s.l, s.rhs, g.stride), kry_norm(Z, nvstride, j, s.l, s.rhs, g.stride),
                        g.stride, i);
#pragma unroll
      for (int c = 0; c < 12; c++) zz[c] = zz[c] - b * a[c];
    }
    WCL_ST(S, ww, w);
    WCL_ST(S, zz, z);
  }
};

// alpha = <w, r> / ||w||^2, aux[4] = 1 / ||w||
template <int S>
struct GcrAlpha {
  FieldRef w, r;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    cpx<typename Traits<S>::R> a[12], b[12];
    WCL_LD(S, true, a, w);
    WCL_LD(S, true, b, r);
    dot_acc(acc, a, b);
    acc[2] += norm_site(a);
  }
  __device__ void finalize(Scalars& c, const double* t) const {
    if (!(t[2] > 0.0)) {
      c.alpha = make_double2(0, 0);
      c.aux[4] = 0.0;
      c.flags |= 1;
    } else {
      c.alpha = make_double2(t[0] / t[2], t[1] / t[2]);
      c.aux[4] = 1.0 / sqrt(t[2]);
    }
  }
};

// x += alpha z; r -= alpha w; then w, z scaled to unit ||w||; r2 = ||r||^2
template <int S, int X>
struct GcrUpdate {
  FieldRef xs, r, w, z;
  const Scalars* sc;
  __device__ void operator()(const Slice& s, const LatGeom& g, long i, double* acc) const {
    using R = typename Traits<S>::R;
    using RX = typename Traits<X>::R;
    const double2 a2 = sc[s.slot].alpha;
    const R inv = R(sc[s.slot].aux[4]);
    const cpx<R> al = {R(a2.x), R(a2.y)};
    const cpx<RX> ax = {RX(a2.x), RX(a2.y)};
    cpx<R> rr[12], ww[12], zz[12];
    cpx<RX> xx[12];
    WCL_LD(S, false, rr, r);
    WCL_LD(S, false, ww, w);
    WCL_LD(S, false, zz, z);
    WCL_LD(X, false, xx, xs);
#pragma unroll
    for (int c = 0; c < 12; c++) {
      xx[c] = xx[c] + ax * cpx<RX>{RX(zz[c].re), RX(zz[c].im)};
      rr[c] = rr[c] - al * ww[c];
      ww[c] = inv * ww[c];
      zz[c] = inv * zz[c];
    }
    WCL_ST(X, xx, xs);
    WCL_ST(S, rr, r);
    WCL_ST(S, ww, w);
    WCL_ST(S, zz, z);
    acc[0] += norm_site(rr);
  }
  __device__ void finalize(Scalars& c, const double* t) const { c.r2 = t[0]; }
};

}  // namespace wcl
