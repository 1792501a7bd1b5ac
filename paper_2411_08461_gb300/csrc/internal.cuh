// Internal types of libwcl: complex arithmetic, per-precision field storage,
// batch geometry (several lattices x several right-hand sides per launch).
//
// Device layouts (all "structure of arrays" so that consecutive threads, which
// own consecutive checkerboard sites, issue coalesced 8/16-byte loads):
//
//   spinor, one parity, one RHS      chunk k of site i at  base[k*stride + i]
//     F64 : 12 chunks of double2 (one complex each, index 3*spin + colour)
//     F32 :  6 chunks of float4  (complexes 2k, 2k+1)
//     F16/BF16 : 3 chunks of uint4 (8 reals each) + float norm[i]
//           (the 24 reals divided by their maximum modulus at the site)
//     RHS r of a field starts at base + r * (nchunk * stride) chunks
//     (norms at norm + r*stride).
//
//   links, per parity p: [mu][chunk][stride]
//     F64 : all 18 reals, 9 double2 (FP64 arithmetic is the scarce resource on
//           GB300, so the FP64 operator skips the row-2 reconstruction)
//     F32 : 12 reals = rows 0 and 1, 3 float4; row 2 rebuilt as conj(row0 x row1)
//     F16/BF16 : the same 12 reals, 3 uint2 (4 reals each, |U_ij| <= 1)
//
//   clover, per parity: two Hermitian 6x6 chiral blocks (spins {0,1} and {2,3},
//     index 3*spin_in_block + colour), each packed as 6 real diagonal entries
//     followed by the 15 complex strictly-lower entries in row-major order:
//     36 reals per block, 72 per site.
//     F64 : 36 double2, F32 : 18 float4, F16/BF16 : 9 uint4 + float norm[i].
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace wcl {

constexpr int MAXLAT = 8;

enum Prec { F64 = 0, F32 = 1, F16 = 2, BF16 = 3, DF64 = 4 };
// DF64: the FP64 fields read into double-float arithmetic (see dfloat below);
// used for intermediate residual replacements, never for a reported result.

// ---------------------------------------------------------------------------
// double-float: value = hi + lo, |lo| <= ulp(hi)/2, a ~48-bit significand on the
// FP32 pipes (Dekker 1971; Knuth's two-sum and the FMA two-product).  On GB300
// FP32 issue is many times the FP64 rate, so this is the cheap way to apply the
// operator with far more than FP32 accuracy.
struct dfloat {
  float hi, lo;
  __host__ __device__ __forceinline__ dfloat() {}
  __host__ __device__ __forceinline__ dfloat(float x) : hi(x), lo(0.f) {}
  __host__ __device__ __forceinline__ dfloat(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ __forceinline__ dfloat(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};
// a stored (hi, lo) pair, already normalised
__host__ __device__ __forceinline__ dfloat df_pair(float hi, float lo) {
  dfloat r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

__device__ __forceinline__ dfloat df_quick(float s, float e) {  // |s| >= |e|
  dfloat r;
  r.hi = __fadd_rn(s, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
  return r;
}
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_quick(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) {
  dfloat r;
  r.hi = -a.hi;
  r.lo = -a.lo;
  return r;
}
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick(p, e);
}
// a * b + c: the exact product of the high parts and its cross terms are added
// to c with one two-sum and one final renormalisation (15 FP32 operations
// instead of 18 for a product followed by a sum)
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  df_two_sum(p, c.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return df_quick(s, t);
}
// keep the floating-point fma visible next to the double-float one
__host__ __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__host__ __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }

template <typename R>
struct cpx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { return cpx<R>{a, b}; }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ cpx<R> cmul_conj(cpx<R> a, cpx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a
template <typename R>
__host__ __device__ __forceinline__ cpx<R> ti(cpx<R> a) { return {-a.im, a.re}; }
// acc += a * b
template <typename R>
__host__ __device__ __forceinline__ void cfma(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ void cfma_conj(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

// ---------------------------------------------------------------------------
// precision traits
template <int P>
struct Traits;
template <>
struct Traits<F64> {
  using R = double;  // compute type
  static constexpr int SP_CHUNK = 12, SP_CHUNK_BYTES = 16;
  static constexpr int LK_CHUNK = 9, LK_CHUNK_BYTES = 16;
  static constexpr int CL_CHUNK = 36, CL_CHUNK_BYTES = 16;
  static constexpr bool HAS_NORM = false;
};
template <>
struct Traits<F32> {
  using R = float;
  static constexpr int SP_CHUNK = 6, SP_CHUNK_BYTES = 16;
  static constexpr int LK_CHUNK = 3, LK_CHUNK_BYTES = 16;
  static constexpr int CL_CHUNK = 18, CL_CHUNK_BYTES = 16;
  static constexpr bool HAS_NORM = false;
};
template <>
struct Traits<F16> {
  using R = float;
  static constexpr int SP_CHUNK = 3, SP_CHUNK_BYTES = 16;
  static constexpr int LK_CHUNK = 3, LK_CHUNK_BYTES = 8;
  static constexpr int CL_CHUNK = 9, CL_CHUNK_BYTES = 16;
  static constexpr bool HAS_NORM = true;
};
template <>
struct Traits<BF16> {
  using R = float;
  static constexpr int SP_CHUNK = 3, SP_CHUNK_BYTES = 16;
  static constexpr int LK_CHUNK = 3, LK_CHUNK_BYTES = 8;
  static constexpr int CL_CHUNK = 9, CL_CHUNK_BYTES = 16;
  static constexpr bool HAS_NORM = true;
};

template <>
struct Traits<DF64> {
  using R = dfloat;  // storage: one float4 (re.hi, re.lo, im.hi, im.lo) per complex
  static constexpr int SP_CHUNK = 12, SP_CHUNK_BYTES = 16;
  static constexpr int LK_CHUNK = 9, LK_CHUNK_BYTES = 16;
  static constexpr int CL_CHUNK = 36, CL_CHUNK_BYTES = 16;
  static constexpr bool HAS_NORM = false;
};

inline int prec_spinor_bytes_per_site(int p) {
  switch (p) {
    case F64:
    case DF64: return 192;
    case F32: return 96;
    default: return 48 + 4;
  }
}

// ---------------------------------------------------------------------------
// 16-bit packing helpers (two reals per 32-bit word)
template <int P>
__device__ __forceinline__ uint32_t pack2(float a, float b);
template <>
__device__ __forceinline__ uint32_t pack2<F16>(float a, float b) {
  __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
template <>
__device__ __forceinline__ uint32_t pack2<BF16>(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}
template <int P>
__device__ __forceinline__ float2 unpack2(uint32_t w);
template <>
__device__ __forceinline__ float2 unpack2<F16>(uint32_t w) {
  return __half22float2(*reinterpret_cast<__half2*>(&w));
}
template <>
__device__ __forceinline__ float2 unpack2<BF16>(uint32_t w) {
  return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&w));
}

// ---------------------------------------------------------------------------
// read-only loads through the non-coherent path
__device__ __forceinline__ double2 ldg(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float4 ldg(const float4* p) { return __ldg(p); }
__device__ __forceinline__ uint4 ldg(const uint4* p) { return __ldg(p); }
__device__ __forceinline__ uint2 ldg(const uint2* p) { return __ldg(p); }
__device__ __forceinline__ float ldg(const float* p) { return __ldg(p); }
// evict-first ("streaming") loads and stores, for data a launch touches once
__device__ __forceinline__ double2 ldcs(const double2* p) { return __ldcs(p); }
__device__ __forceinline__ float4 ldcs(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ldcs(const uint4* p) { return __ldcs(p); }
__device__ __forceinline__ uint2 ldcs(const uint2* p) { return __ldcs(p); }
__device__ __forceinline__ float ldcs(const float* p) { return __ldcs(p); }
template <bool CS, typename T>
__device__ __forceinline__ T ldp(const T* p) {
  if (CS) return ldcs(p);
  return ldg(p);
}
template <bool CS, typename T>
__device__ __forceinline__ void stp(T* p, const T& v) {
  if (CS)
    __stcs(p, v);
  else
    *p = v;
}
// NC = true: non-coherent read-only path (field not written by this kernel);
// NC = false: ordinary load (field updated in place by the same kernel).
template <bool NC, typename T>
__device__ __forceinline__ T ld(const T* p) {
  if (NC) return ldg(p);
  return *p;
}

// ---------------------------------------------------------------------------
// spinor access: 12 complexes (index 3*spin + colour) at site i
template <int P>
struct SpinorIO;

template <>
struct SpinorIO<F64> {
  using R = double;
  template <bool NC = true>
  __device__ static void load(cpx<R> v[12], const void* base, const float*, long stride, long i) {
    const double2* p = static_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      double2 d = ld<NC>(p + k * stride + i);
      v[k] = {d.x, d.y};
    }
  }
  template <bool CS = false>
  __device__ static void store(const cpx<R> v[12], void* base, float*, long stride, long i) {
    double2* p = static_cast<double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) stp<CS>(p + k * stride + i, make_double2(v[k].re, v[k].im));
  }
  __device__ static void load_cs(cpx<R> v[12], const void* base, const float*, long stride, long i) {
    const double2* p = static_cast<const double2*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double2 d = ldcs(p + k * stride + i);
      v[k] = {d.x, d.y};
    }
  }
};

template <>
struct SpinorIO<DF64> {
  using R = dfloat;
  template <bool NC = true>
  __device__ static void load(cpx<R> v[12], const void* base, const float*, long stride, long i) {
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const float4 f = ld<NC>(p + k * stride + i);
      v[k] = {df_pair(f.x, f.y), df_pair(f.z, f.w)};
    }
  }
  __device__ static void store(const cpx<R> v[12], void* base, float*, long stride, long i) {
    float4* p = static_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 12; k++) p[k * stride + i] = make_float4(v[k].re.hi, v[k].re.lo, v[k].im.hi, v[k].im.lo);
  }
};

template <>
struct SpinorIO<F32> {
  using R = float;
  template <bool NC = true>
  __device__ static void load(cpx<R> v[12], const void* base, const float*, long stride, long i) {
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 f = ld<NC>(p + k * stride + i);
      v[2 * k] = {f.x, f.y};
      v[2 * k + 1] = {f.z, f.w};
    }
  }
  template <bool CS = false>
  __device__ static void store(const cpx<R> v[12], void* base, float*, long stride, long i) {
    float4* p = static_cast<float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++)
      stp<CS>(p + k * stride + i, make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im));
  }
  __device__ static void load_cs(cpx<R> v[12], const void* base, const float*, long stride, long i) {
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float4 f = ldcs(p + k * stride + i);
      v[2 * k] = {f.x, f.y};
      v[2 * k + 1] = {f.z, f.w};
    }
  }
};

template <int P>
struct SpinorIO16 {
  using R = float;
  template <bool NC = true>
  __device__ static void load(cpx<R> v[12], const void* base, const float* norm, long stride, long i) {
    const uint4* p = static_cast<const uint4*>(base);
    float n = ld<NC>(norm + i);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 q = ld<NC>(p + k * stride + i);
      float2 a = unpack2<P>(q.x), b = unpack2<P>(q.y), c = unpack2<P>(q.z), d = unpack2<P>(q.w);
      v[4 * k + 0] = {a.x * n, a.y * n};
      v[4 * k + 1] = {b.x * n, b.y * n};
      v[4 * k + 2] = {c.x * n, c.y * n};
      v[4 * k + 3] = {d.x * n, d.y * n};
    }
  }
  template <bool CS = false>
  __device__ static void store(const cpx<R> v[12], void* base, float* norm, long stride, long i) {
    uint4* p = static_cast<uint4*>(base);
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(v[k].re), fabsf(v[k].im)));
    float inv = m > 0.f ? 1.0f / m : 0.f;
    stp<CS>(norm + i, m);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 q;
      q.x = pack2<P>(v[4 * k + 0].re * inv, v[4 * k + 0].im * inv);
      q.y = pack2<P>(v[4 * k + 1].re * inv, v[4 * k + 1].im * inv);
      q.z = pack2<P>(v[4 * k + 2].re * inv, v[4 * k + 2].im * inv);
      q.w = pack2<P>(v[4 * k + 3].re * inv, v[4 * k + 3].im * inv);
      stp<CS>(p + k * stride + i, q);
    }
  }
  __device__ static void load_cs(cpx<R> v[12], const void* base, const float* norm, long stride, long i) {
    const uint4* p = static_cast<const uint4*>(base);
    const float n = ldcs(norm + i);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint4 q = ldcs(p + k * stride + i);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int m = 0; m < 4; m++) {
        const float2 f = unpack2<P>(w[m]);
        v[4 * k + m] = {f.x * n, f.y * n};
      }
    }
  }
};
template <>
struct SpinorIO<F16> : SpinorIO16<F16> {};
template <>
struct SpinorIO<BF16> : SpinorIO16<BF16> {};

// ---------------------------------------------------------------------------
// link access: U_mu at site i of one parity block [mu][chunk][stride]
template <int P>
struct LinkIO;

template <typename R>
__device__ __forceinline__ void reconstruct_row2(cpx<R> u[3][3]) {
  // row2 = conj(row0 x row1)
  u[2][0] = conj(u[0][1] * u[1][2] - u[0][2] * u[1][1]);
  u[2][1] = conj(u[0][2] * u[1][0] - u[0][0] * u[1][2]);
  u[2][2] = conj(u[0][0] * u[1][1] - u[0][1] * u[1][0]);
}

template <>
struct LinkIO<F64> {
  using R = double;
  template <bool CS = false>
  __device__ static void load(cpx<R> u[3][3], const void* base, long stride, long i, int mu) {
    const double2* p = static_cast<const double2*>(base) + (long)mu * 9 * stride;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      double2 d = ldp<CS>(p + k * stride + i);
      u[k / 3][k % 3] = {d.x, d.y};
    }
  }
};
template <>
struct LinkIO<DF64> {
  using R = dfloat;
  __device__ static void load(cpx<R> u[3][3], const void* base, long stride, long i, int mu) {
    const float4* p = static_cast<const float4*>(base) + (long)mu * 9 * stride;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const float4 f = ldg(p + k * stride + i);
      u[k / 3][k % 3] = {df_pair(f.x, f.y), df_pair(f.z, f.w)};
    }
  }
};
template <>
struct LinkIO<F32> {
  using R = float;
  template <bool CS = false>
  __device__ static void load(cpx<R> u[3][3], const void* base, long stride, long i, int mu) {
    const float4* p = static_cast<const float4*>(base) + (long)mu * 3 * stride;
    float4 a = ldp<CS>(p + i), b = ldp<CS>(p + stride + i), c = ldp<CS>(p + 2 * stride + i);
    u[0][0] = {a.x, a.y};
    u[0][1] = {a.z, a.w};
    u[0][2] = {b.x, b.y};
    u[1][0] = {b.z, b.w};
    u[1][1] = {c.x, c.y};
    u[1][2] = {c.z, c.w};
    reconstruct_row2(u);
  }
};
template <int P>
struct LinkIO16 {
  using R = float;
  template <bool CS = false>
  __device__ static void load(cpx<R> u[3][3], const void* base, long stride, long i, int mu) {
    const uint2* p = static_cast<const uint2*>(base) + (long)mu * 3 * stride;
    uint2 a = ldp<CS>(p + i), b = ldp<CS>(p + stride + i), c = ldp<CS>(p + 2 * stride + i);
    float2 t;
    t = unpack2<P>(a.x); u[0][0] = {t.x, t.y};
    t = unpack2<P>(a.y); u[0][1] = {t.x, t.y};
    t = unpack2<P>(b.x); u[0][2] = {t.x, t.y};
    t = unpack2<P>(b.y); u[1][0] = {t.x, t.y};
    t = unpack2<P>(c.x); u[1][1] = {t.x, t.y};
    t = unpack2<P>(c.y); u[1][2] = {t.x, t.y};
    reconstruct_row2(u);
  }
};
template <>
struct LinkIO<F16> : LinkIO16<F16> {};
template <>
struct LinkIO<BF16> : LinkIO16<BF16> {};

// ---------------------------------------------------------------------------
// clover: y = C x for the two Hermitian 6x6 chiral blocks at site i.
// Packed block: d[0..5] real diagonal, then L[k] complex, k = r(r-1)/2 + c for r > c.
template <typename R>
__device__ __forceinline__ void hermitian6_apply(cpx<R> y[6], const R d[6], const cpx<R> L[15], const cpx<R> x[6]) {
#pragma unroll
  for (int r = 0; r < 6; r++) y[r] = d[r] * x[r];
#pragma unroll
  for (int r = 1; r < 6; r++) {
#pragma unroll
    for (int c = 0; c < r; c++) {
      const cpx<R> l = L[r * (r - 1) / 2 + c];
      cfma(y[r], l, x[c]);       // lower entry (r, c)
      cfma_conj(y[c], l, x[r]);  // upper entry (c, r) = conj(l)
    }
  }
}

template <int P>
struct CloverIO;

template <>
struct CloverIO<F64> {
  using R = double;
  __device__ static void apply(cpx<R> y[12], const cpx<R> x[12], const void* base, const float*, long stride, long i) {
    const double2* p = static_cast<const double2*>(base);
#pragma unroll
    for (int b = 0; b < 2; b++) {
      R d[6];
      cpx<R> L[15];
#pragma unroll
      for (int k = 0; k < 3; k++) {
        double2 v = ldg(p + (18 * b + k) * stride + i);
        d[2 * k] = v.x;
        d[2 * k + 1] = v.y;
      }
#pragma unroll
      for (int k = 0; k < 15; k++) {
        double2 v = ldg(p + (18 * b + 3 + k) * stride + i);
        L[k] = {v.x, v.y};
      }
      hermitian6_apply(y + 6 * b, d, L, x + 6 * b);
    }
  }
};
template <>
struct CloverIO<DF64> {
  using R = dfloat;
  __device__ static void apply(cpx<R> y[12], const cpx<R> x[12], const void* base, const float*, long stride, long i) {
    const float4* p = static_cast<const float4*>(base);
    // one copy of the block multiply (code size: the double-float kernels are
    // bound by instruction fetch when fully unrolled)
#pragma unroll 1
    for (int b = 0; b < 2; b++) {
      R d[6];
      cpx<R> L[15];
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const float4 f = ldg(p + (18 * b + k) * stride + i);
        d[2 * k] = df_pair(f.x, f.y);
        d[2 * k + 1] = df_pair(f.z, f.w);
      }
#pragma unroll
      for (int k = 0; k < 15; k++) {
        const float4 f = ldg(p + (18 * b + 3 + k) * stride + i);
        L[k] = {df_pair(f.x, f.y), df_pair(f.z, f.w)};
      }
      hermitian6_apply(y + 6 * b, d, L, x + 6 * b);
    }
  }
};
template <>
struct CloverIO<F32> {
  using R = float;
  __device__ static void apply(cpx<R> y[12], const cpx<R> x[12], const void* base, const float*, long stride, long i) {
    const float4* p = static_cast<const float4*>(base);
#pragma unroll
    for (int b = 0; b < 2; b++) {
      float r[36];
#pragma unroll
      for (int k = 0; k < 9; k++) {
        float4 v = ldg(p + (9 * b + k) * stride + i);
        r[4 * k] = v.x;
        r[4 * k + 1] = v.y;
        r[4 * k + 2] = v.z;
        r[4 * k + 3] = v.w;
      }
      R d[6];
      cpx<R> L[15];
#pragma unroll
      for (int k = 0; k < 6; k++) d[k] = r[k];
#pragma unroll
      for (int k = 0; k < 15; k++) L[k] = {r[6 + 2 * k], r[7 + 2 * k]};
      hermitian6_apply(y + 6 * b, d, L, x + 6 * b);
    }
  }
};
template <int P>
struct CloverIO16 {
  using R = float;
  __device__ static void apply(cpx<R> y[12], const cpx<R> x[12], const void* base, const float* norm, long stride, long i) {
    const uint4* p = static_cast<const uint4*>(base);
    const float n = __ldg(norm + i);
    float r[72];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      uint4 q = ldg(p + k * stride + i);
      float2 a = unpack2<P>(q.x), b = unpack2<P>(q.y), c = unpack2<P>(q.z), d = unpack2<P>(q.w);
      r[8 * k + 0] = a.x * n; r[8 * k + 1] = a.y * n;
      r[8 * k + 2] = b.x * n; r[8 * k + 3] = b.y * n;
      r[8 * k + 4] = c.x * n; r[8 * k + 5] = c.y * n;
      r[8 * k + 6] = d.x * n; r[8 * k + 7] = d.y * n;
    }
#pragma unroll
    for (int b = 0; b < 2; b++) {
      R d[6];
      cpx<R> L[15];
#pragma unroll
      for (int k = 0; k < 6; k++) d[k] = r[36 * b + k];
#pragma unroll
      for (int k = 0; k < 15; k++) L[k] = {r[36 * b + 6 + 2 * k], r[36 * b + 7 + 2 * k]};
      hermitian6_apply(y + 6 * b, d, L, x + 6 * b);
    }
  }
};
template <>
struct CloverIO<F16> : CloverIO16<F16> {};
template <>
struct CloverIO<BF16> : CloverIO16<BF16> {};

// ---------------------------------------------------------------------------
// Batch geometry: one launch covers several lattices, each with nrhs
// right-hand sides.  Blocks are assigned lattice by lattice; inside a lattice
// the RHS index varies fastest so that the blocks working on the same sites for
// different RHS run together and share links and clover through L1/L2.
struct LatGeom {
  int dims[4];      // Lx, Ly, Lz, Lt
  int lxh;          // Lx / 2
  int vh;           // sites per parity
  long stride;      // padded sites per chunk
  int nrhs;
  int block_begin;  // first block of this lattice in the launch
  int nchunk;       // site blocks per RHS
  int slot_base;    // index of (lattice, rhs = 0) in per-slice arrays
  float tb;         // fermion time boundary sign
  int zblk;         // multi-RHS kernel: z planes per block of its tile order (0: tiles in site order)
  double tw;        // weight of the t hops relative to the spatial ones (xi_0 / nu; 1 isotropic)
  float tw_f;       // tw and tb * tw rounded to FP32 for the FP32 / 16-bit kernels
  float tbw_f;
};

// factor of a t hop: tw inside the lattice, tb * tw across the time boundary
template <typename R>
__device__ __forceinline__ R hop_t_weight(const LatGeom& g, bool edge) {
  if constexpr (std::is_same<R, double>::value) {
    return edge ? (double)g.tb * g.tw : g.tw;
  } else if constexpr (std::is_same<R, float>::value) {
    return edge ? g.tbw_f : g.tw_f;
  } else {
    return R(edge ? (double)g.tb * g.tw : g.tw);  // double-float: split once per thread
  }
}

struct Batch {
  int nlat;
  int total_blocks;
  LatGeom lat[MAXLAT];
};

struct Slice {
  int l;       // lattice
  int rhs;     // right-hand side
  int chunk;   // block index within the (lattice, rhs) slice
  int slot;    // slot_base + rhs
};

__device__ __forceinline__ Slice find_slice(const Batch& b, int block) {
  int l = 0;
#pragma unroll 1
  for (int k = 1; k < b.nlat; k++)
    if (block >= b.lat[k].block_begin) l = k;
  const LatGeom& g = b.lat[l];
  int local = block - g.block_begin;
  Slice s;
  s.l = l;
  s.rhs = local % g.nrhs;
  s.chunk = local / g.nrhs;
  s.slot = g.slot_base + s.rhs;
  return s;
}

// A field on every lattice of a batch: per-lattice base pointers, RHS stacked.
struct FieldRef {
  void* ptr[MAXLAT];
  float* norm[MAXLAT];
};

template <int P>
__device__ __forceinline__ const void* rhs_ptr(const FieldRef& f, int l, int rhs, long stride) {
  return static_cast<const char*>(f.ptr[l]) + (size_t)rhs * Traits<P>::SP_CHUNK * Traits<P>::SP_CHUNK_BYTES * stride;
}
template <int P>
__device__ __forceinline__ void* rhs_ptr_w(const FieldRef& f, int l, int rhs, long stride) {
  return static_cast<char*>(f.ptr[l]) + (size_t)rhs * Traits<P>::SP_CHUNK * Traits<P>::SP_CHUNK_BYTES * stride;
}
__device__ __forceinline__ float* rhs_norm(const FieldRef& f, int l, int rhs, long stride) {
  return f.norm[l] ? f.norm[l] + (size_t)rhs * stride : nullptr;
}

// Per-(lattice, rhs) solver scalars, kept on the device so that the solver
// iterations need no host round trip.
struct Scalars {
  double2 rho, rho_prev, alpha, omega, beta;
  double r2;       // ||r||^2 of the iterated residual
  double r2_prev;
  double aux[6];   // scratch for finalizers
  int flags;       // bit 0: breakdown seen
  int pad;
};

}  // namespace wcl
