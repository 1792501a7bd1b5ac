// Multi-RHS fused dslash + clover on packed FP32 pairs (Blackwell FFMA2 / FADD2).
//
// Same operator and modes as dslash_mrhs_kernel (out = C_post(alpha D in + beta C_pre x),
// Eq. 5's hopping term with the clover term fused, several right-hand sides per CTA),
// with the arithmetic reorganised for sm_100+: every thread owns one site and a PAIR
// of right-hand sides (2q, 2q + 1), and keeps each real component of the two
// right-hand sides in one float2 register pair -- .x for RHS 2q, .y for RHS 2q + 1 --
// so that one packed instruction (__ffma2_rn, __fadd2_rn, __fmul2_rn) does the work
// of two FP32 ones.  The link and clover entries, shared by both right-hand sides,
// are stored duplicated in shared memory, (u, u) per real, so that a 16-byte read
// gives (re, re, im, im) of one complex entry ready for the packed multiply.
//
// Spinors stay in the library's per-RHS layout; the spin projection and the 16-bit
// decoding are scalar and write straight into the lanes of the packed registers,
// the link multiply, the spin reconstruction and the clover multiply are packed.
// Multiplying a packed complex number by i costs nothing: it swaps the roles of its
// re and im registers.
#pragma once
#include "dslash.cuh"

namespace wcl {

// a complex number of two right-hand sides
struct c2 {
  float2 re, im;
};

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_neg(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }

// Shared-memory rows (floats): a link is its 18 reals each stored twice (36 floats;
// 36 mod 32 = 4, so consecutive sites' 16-byte reads fall in distinct banks); the
// clover pair of blocks is its 72 reals each stored twice, padded to 148.
constexpr int PAIR_LROW = 36, PAIR_CROW = 148;

// o = sign U h (ADJ: sign U^+ h) on both spin halves; U from its duplicated row
template <bool ADJ>
__device__ __forceinline__ void pair_link_mul(const float* row, const c2 h[6], c2 o[6], float2 sign) {
  // the negated factor of each complex product: -Im h for U h, -Re h for U^+ h
  float2 nh[6];
#pragma unroll
  for (int k = 0; k < 6; k++) nh[k] = p_neg(ADJ ? h[k].re : h[k].im);
#pragma unroll
  for (int e = 0; e < 9; e++) {
    const int a = e / 3, b = e % 3;
    const float4 u = reinterpret_cast<const float4*>(row)[e];  // (re, re, im, im)
    const float2 ur = make_float2(u.x, u.y), ui = make_float2(u.z, u.w);
#pragma unroll
    for (int k = 0; k < 2; k++) {
      if (!ADJ) {  // o_a += U_ab h_b
        const c2& x = h[3 * k + b];
        c2& y = o[3 * k + a];
        if (b == 0) {
          y.re = p_mul(ur, x.re);
          y.im = p_mul(ur, x.im);
        } else {
          y.re = p_fma(ur, x.re, y.re);
          y.im = p_fma(ur, x.im, y.im);
        }
        y.re = p_fma(ui, nh[3 * k + b], y.re);
        y.im = p_fma(ui, x.re, y.im);
      } else {  // o_b += conj(U_ab) h_a
        const c2& x = h[3 * k + a];
        c2& y = o[3 * k + b];
        if (a == 0) {
          y.re = p_mul(ur, x.re);
          y.im = p_mul(ur, x.im);
        } else {
          y.re = p_fma(ur, x.re, y.re);
          y.im = p_fma(ur, x.im, y.im);
        }
        y.re = p_fma(ui, x.im, y.re);
        y.im = p_fma(ui, nh[3 * k + a], y.im);
      }
    }
  }
  if (sign.x != 1.f || sign.y != 1.f) {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      o[k].re = p_mul(sign, o[k].re);
      o[k].im = p_mul(sign, o[k].im);
    }
  }
}

// acc += reconstruction of the two-spinor o for hop direction MU with projector sign S
// (the same table as reconstruct_acc; i * z has re = -z.im, im = z.re)
template <int MU, int S>
__device__ __forceinline__ void pair_reconstruct(c2 acc[12], const c2 o[6]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const c2 h0 = o[c], h1 = o[3 + c];
    acc[c].re = p_add(acc[c].re, h0.re);
    acc[c].im = p_add(acc[c].im, h0.im);
    acc[3 + c].re = p_add(acc[3 + c].re, h1.re);
    acc[3 + c].im = p_add(acc[3 + c].im, h1.im);
    c2& l2 = acc[6 + c];
    c2& l3 = acc[9 + c];
    if (MU == 0) {  // S>0: l2 -= i h1, l3 -= i h0
      if (S > 0) {
        l2.re = p_add(l2.re, h1.im); l2.im = p_sub(l2.im, h1.re);
        l3.re = p_add(l3.re, h0.im); l3.im = p_sub(l3.im, h0.re);
      } else {
        l2.re = p_sub(l2.re, h1.im); l2.im = p_add(l2.im, h1.re);
        l3.re = p_sub(l3.re, h0.im); l3.im = p_add(l3.im, h0.re);
      }
    } else if (MU == 1) {  // S>0: l2 += h1, l3 -= h0
      if (S > 0) {
        l2.re = p_add(l2.re, h1.re); l2.im = p_add(l2.im, h1.im);
        l3.re = p_sub(l3.re, h0.re); l3.im = p_sub(l3.im, h0.im);
      } else {
        l2.re = p_sub(l2.re, h1.re); l2.im = p_sub(l2.im, h1.im);
        l3.re = p_add(l3.re, h0.re); l3.im = p_add(l3.im, h0.im);
      }
    } else if (MU == 2) {  // S>0: l2 -= i h0, l3 += i h1
      if (S > 0) {
        l2.re = p_add(l2.re, h0.im); l2.im = p_sub(l2.im, h0.re);
        l3.re = p_sub(l3.re, h1.im); l3.im = p_add(l3.im, h1.re);
      } else {
        l2.re = p_sub(l2.re, h0.im); l2.im = p_add(l2.im, h0.re);
        l3.re = p_add(l3.re, h1.im); l3.im = p_sub(l3.im, h1.re);
      }
    } else {  // S>0: l2 += h0, l3 += h1
      if (S > 0) {
        l2.re = p_add(l2.re, h0.re); l2.im = p_add(l2.im, h0.im);
        l3.re = p_add(l3.re, h1.re); l3.im = p_add(l3.im, h1.im);
      } else {
        l2.re = p_sub(l2.re, h0.re); l2.im = p_sub(l2.im, h0.im);
        l3.re = p_sub(l3.re, h1.re); l3.im = p_sub(l3.im, h1.im);
      }
    }
  }
}

// spin projection of two right-hand sides' spinors into one packed half spinor
template <int MU, int S>
__device__ __forceinline__ void pair_project(const cpx<float> p[12], const cpx<float> q[12], c2 h[6]) {
  cpx<float> a[6], b[6];
  project<MU, S>(p, a);
  project<MU, S>(q, b);
#pragma unroll
  for (int k = 0; k < 6; k++) {
    h[k].re = make_float2(a[k].re, b[k].re);
    h[k].im = make_float2(a[k].im, b[k].im);
  }
}

// y = C x for one Hermitian 6x6 block from its duplicated row (6 diagonal reals, then
// the 15 lower entries as (re, re, im, im)), same order of operations as
// hermitian6_apply_row
__device__ __forceinline__ void pair_hermitian6(c2 y[6], const float* row, const c2 x[6]) {
  c2 nx[6];
#pragma unroll
  for (int r = 0; r < 6; r++) {
    nx[r].re = p_neg(x[r].re);
    nx[r].im = p_neg(x[r].im);
  }
#pragma unroll
  for (int r = 0; r < 6; r++) {
    const float2 d = reinterpret_cast<const float2*>(row)[r];
    y[r].re = p_mul(d, x[r].re);
    y[r].im = p_mul(d, x[r].im);
  }
#pragma unroll
  for (int k = 0; k < 15; k++) {
    const int r = tri_row(k), c = tri_col(k);
    const float4 l = reinterpret_cast<const float4*>(row + 12)[k];
    const float2 lr = make_float2(l.x, l.y), li = make_float2(l.z, l.w);
    // lower entry (r, c): y_r += l x_c
    y[r].re = p_fma(lr, x[c].re, y[r].re);
    y[r].re = p_fma(li, nx[c].im, y[r].re);
    y[r].im = p_fma(lr, x[c].im, y[r].im);
    y[r].im = p_fma(li, x[c].re, y[r].im);
    // upper entry (c, r) = conj(l): y_c += conj(l) x_r
    y[c].re = p_fma(lr, x[r].re, y[c].re);
    y[c].re = p_fma(li, x[r].im, y[c].re);
    y[c].im = p_fma(lr, x[r].im, y[c].im);
    y[c].im = p_fma(li, nx[r].re, y[c].im);
  }
}

// y += beta C x for one block (beta folded into C's entries, as hermitian6_axpy_row)
__device__ __forceinline__ void pair_hermitian6_axpy(c2 y[6], float beta, const float* row, const c2 x[6]) {
  const float2 b2 = make_float2(beta, beta);
  c2 nx[6];
#pragma unroll
  for (int r = 0; r < 6; r++) {
    nx[r].re = p_neg(x[r].re);
    nx[r].im = p_neg(x[r].im);
  }
#pragma unroll
  for (int r = 0; r < 6; r++) {
    const float2 d = p_mul(b2, reinterpret_cast<const float2*>(row)[r]);
    y[r].re = p_fma(d, x[r].re, y[r].re);
    y[r].im = p_fma(d, x[r].im, y[r].im);
  }
#pragma unroll
  for (int k = 0; k < 15; k++) {
    const int r = tri_row(k), c = tri_col(k);
    const float4 l = reinterpret_cast<const float4*>(row + 12)[k];
    const float2 lr = p_mul(b2, make_float2(l.x, l.y)), li = p_mul(b2, make_float2(l.z, l.w));
    y[r].re = p_fma(lr, x[c].re, y[r].re);
    y[r].re = p_fma(li, nx[c].im, y[r].re);
    y[r].im = p_fma(lr, x[c].im, y[r].im);
    y[r].im = p_fma(li, x[c].re, y[r].im);
    y[c].re = p_fma(lr, x[r].re, y[c].re);
    y[c].re = p_fma(li, x[r].im, y[c].re);
    y[c].im = p_fma(lr, x[r].im, y[c].im);
    y[c].im = p_fma(li, nx[r].re, y[c].im);
  }
}

// the two right-hand sides of a pair as ordinary complex spinors (for stores and sums)
__device__ __forceinline__ void pair_split(const c2 v[12], cpx<float> a[12], cpx<float> b[12]) {
#pragma unroll
  for (int k = 0; k < 12; k++) {
    a[k] = {v[k].re.x, v[k].im.x};
    b[k] = {v[k].re.y, v[k].im.y};
  }
}
__device__ __forceinline__ void pair_join(const cpx<float> a[12], const cpx<float> b[12], c2 v[12]) {
#pragma unroll
  for (int k = 0; k < 12; k++) {
    v[k].re = make_float2(a[k].re, b[k].re);
    v[k].im = make_float2(a[k].im, b[k].im);
  }
}

template <int MU, bool BACK, bool DAG, int P>
__device__ __forceinline__ void pair_hop(c2 acc[12], const void* in0, const void* in1, const float* n0,
                                         const float* n1, long stride, long j, const float* U, float2 sign) {
  constexpr int SF = DAG ? +1 : -1;
  constexpr int S = BACK ? -SF : SF;
  c2 h[6], o[6];
  {
    cpx<float> p[12], q[12];
    SpinorIO<P>::load(p, in0, n0, stride, j);
    SpinorIO<P>::load(q, in1, n1, stride, j);
    pair_project<MU, S>(p, q, h);
  }
  pair_link_mul<BACK>(U, h, o, sign);
  pair_reconstruct<MU, S>(acc, o);
}

// Pair kernel bounds: TS sites x up to 8 pairs (16 RHS) per CTA.
template <int TS>
struct PairBounds;
// Every variant is given 128 registers per thread (the packed accumulators of two
// right-hand sides alone take 48); with 12 RHS that is 10 / 5 / 2 CTAs of 64 / 96 /
// 192 threads per SM.
template <>
struct PairBounds<8> {
  static constexpr int THREADS = 64, MIN_BLOCKS = 8;
};
template <>
struct PairBounds<16> {
  static constexpr int THREADS = 128, MIN_BLOCKS = 4;
};
template <>
struct PairBounds<32> {
  static constexpr int THREADS = 256, MIN_BLOCKS = 2;
};

// tile of a multi-RHS CTA in the (optionally z-blocked) tile order of dslash_mrhs_kernel
__device__ __forceinline__ long mrhs_tile(const LatGeom& g, long tile, int ts) {
  if (g.zblk <= 0) return tile;
  const int tpr = g.lxh / ts, Ly = g.dims[1], Lz = g.dims[2], Lt = g.dims[3], bz = g.zblk;
  long q = tile;
  const int xt = (int)(q % tpr);
  q /= tpr;
  const int y = (int)(q % Ly);
  q /= Ly;
  const int zz = (int)(q % bz);
  q /= bz;
  const int t = (int)(q % Lt);
  const int zb = (int)(q / Lt);
  return (((long)t * Lz + zb * bz + zz) * Ly + y) * tpr + xt;
}

template <int P, bool DAG, int MODE, int EPI, int TS>
__global__ void __launch_bounds__(PairBounds<TS>::THREADS, PairBounds<TS>::MIN_BLOCKS)
    dslash_pair_kernel(const __grid_constant__ DslashArgs a) {
  constexpr bool CLOV = (MODE & MODE_POST) || (MODE & MODE_PRE);
  extern __shared__ __align__(16) float pair_smem[];
  float* Us = pair_smem;                        // [8][TS][PAIR_LROW]
  float* Cs = Us + 8 * TS * PAIR_LROW;          // [TS][PAIR_CROW]
  __shared__ int Nb[8][TS];
  __shared__ unsigned char Tb[TS];
  const Slice s = find_slice(a.b, blockIdx.x);  // one slice per lattice
  const LatGeom& g = a.b.lat[s.l];
  const int nrhs = a.nrhs_tc;
  const int slot0 = s.l * nrhs;
  const int p = a.out_parity;
  const long stride = g.stride;
  const long site0 = mrhs_tile(g, s.chunk, TS) * TS;

  // phase 0: neighbours of the tile's sites
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
  // phase 1: links (row 2 rebuilt, 16-bit scaled) and clover of the tile, every real twice
  for (int e = threadIdx.x; e < 8 * TS; e += blockDim.x) {
    const int ls = e % TS, d = e / TS, mu = d >> 1;
    const long i = site0 + ls;
    cpx<float> u[3][3];
    if (i < g.vh) {
      if (d & 1)
        LinkIO<P>::template load<true>(u, a.gauge[s.l][1 - p], stride, Nb[d][ls], mu);
      else
        LinkIO<P>::template load<true>(u, a.gauge[s.l][p], stride, i, mu);
    } else {
#pragma unroll
      for (int k = 0; k < 9; k++) u[k / 3][k % 3] = {0.f, 0.f};
    }
    float4* row = reinterpret_cast<float4*>(Us + (d * TS + ls) * PAIR_LROW);
#pragma unroll
    for (int k = 0; k < 9; k++) row[k] = make_float4(u[k / 3][k % 3].re, u[k / 3][k % 3].re, u[k / 3][k % 3].im,
                                                     u[k / 3][k % 3].im);
  }
  if (CLOV) {
    using CC = CloverChunk<P>;
    const void* cb = (MODE & MODE_POST) ? a.cpost[s.l] : a.cpre[s.l];
    const float* cn = (MODE & MODE_POST) ? a.cpost_norm[s.l] : a.cpre_norm[s.l];
    for (int e = threadIdx.x; e < CC::NCH * TS; e += blockDim.x) {
      const int ls = e % TS, k = e / TS;
      const long i = site0 + ls;
      float r[CC::PER];
      if (i < g.vh) {
        CC::load(r, cb, cn, stride, i, k);
      } else {
#pragma unroll
        for (int j = 0; j < CC::PER; j++) r[j] = 0.f;
      }
      float2* row = reinterpret_cast<float2*>(Cs + ls * PAIR_CROW);
#pragma unroll
      for (int j = 0; j < CC::PER; j++) row[CC::PER * k + j] = make_float2(r[j], r[j]);
    }
  }
  __syncthreads();

  // phase 2: thread = (site ls, pair q); the TS threads of one pair are consecutive lanes
  const int ls = threadIdx.x % TS, q = threadIdx.x / TS;
  const int r0 = 2 * q, r1 = (2 * q + 1 < nrhs) ? 2 * q + 1 : 2 * q;  // odd count: last pair doubled
  const long i = site0 + ls;
  const bool act0 = r0 < nrhs && (!a.active || a.active[slot0 + r0]);
  const bool act1 = 2 * q + 1 < nrhs && (!a.active || a.active[slot0 + r1]);
  double red0[3] = {0.0, 0.0, 0.0}, red1[3] = {0.0, 0.0, 0.0};
  if ((act0 || act1) && i < g.vh) {
    const void* in0 = rhs_ptr<P>(a.in, s.l, r0, stride);
    const void* in1 = rhs_ptr<P>(a.in, s.l, r1, stride);
    const float* n0 = rhs_norm(a.in, s.l, r0, stride);
    const float* n1 = rhs_norm(a.in, s.l, r1, stride);
    c2 acc[12];
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k].re = acc[k].im = make_float2(0.f, 0.f);
    const int tb = Tb[ls];
    const float sfv = hop_t_weight<float>(g, tb & 1), sbv = hop_t_weight<float>(g, tb & 2);
    const float2 one = make_float2(1.f, 1.f);
    const float* U0 = Us + ls * PAIR_LROW;
    constexpr int LS = TS * PAIR_LROW;  // floats between the rows of two directions
    pair_hop<0, false, DAG, P>(acc, in0, in1, n0, n1, stride, Nb[0][ls], U0 + 0 * LS, one);
    pair_hop<0, true, DAG, P>(acc, in0, in1, n0, n1, stride, Nb[1][ls], U0 + 1 * LS, one);
    pair_hop<1, false, DAG, P>(acc, in0, in1, n0, n1, stride, Nb[2][ls], U0 + 2 * LS, one);
    pair_hop<1, true, DAG, P>(acc, in0, in1, n0, n1, stride, Nb[3][ls], U0 + 3 * LS, one);
    pair_hop<2, false, DAG, P>(acc, in0, in1, n0, n1, stride, Nb[4][ls], U0 + 4 * LS, one);
    pair_hop<2, true, DAG, P>(acc, in0, in1, n0, n1, stride, Nb[5][ls], U0 + 5 * LS, one);
    pair_hop<3, false, DAG, P>(acc, in0, in1, n0, n1, stride, Nb[6][ls], U0 + 6 * LS, make_float2(sfv, sfv));
    pair_hop<3, true, DAG, P>(acc, in0, in1, n0, n1, stride, Nb[7][ls], U0 + 7 * LS, make_float2(sbv, sbv));
    const float al = (float)a.alpha[s.l];
    const float2 alpha = make_float2(al, al);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      acc[k].re = p_mul(alpha, acc[k].re);
      acc[k].im = p_mul(alpha, acc[k].im);
    }
    const float* crow = Cs + ls * PAIR_CROW;
    if (MODE & MODE_XPAY) {
      c2 xv[12];
      {
        cpx<float> x0[12], x1[12];
        SpinorIO<P>::load_cs(x0, rhs_ptr<P>(a.x, s.l, r0, stride), rhs_norm(a.x, s.l, r0, stride), stride, i);
        SpinorIO<P>::load_cs(x1, rhs_ptr<P>(a.x, s.l, r1, stride), rhs_norm(a.x, s.l, r1, stride), stride, i);
        pair_join(x0, x1, xv);
      }
      const float beta = (float)a.beta[s.l];
      if (MODE & MODE_PRE) {
        pair_hermitian6_axpy(acc, beta, crow, xv);
        pair_hermitian6_axpy(acc + 6, beta, crow + 72, xv + 6);
      } else {
        const float2 b2 = make_float2(beta, beta);
#pragma unroll
        for (int k = 0; k < 12; k++) {
          acc[k].re = p_fma(b2, xv[k].re, acc[k].re);
          acc[k].im = p_fma(b2, xv[k].im, acc[k].im);
        }
      }
      if (EPI != EPI_NONE) {
        cpx<float> o0[12], o1[12], f0[12], f1[12];
        pair_split(acc, o0, o1);
        if (EPI == EPI_ALPHA) {
          SpinorIO<P>::load_cs(f0, rhs_ptr<P>(a.f, s.l, r0, stride), rhs_norm(a.f, s.l, r0, stride), stride, i);
          SpinorIO<P>::load_cs(f1, rhs_ptr<P>(a.f, s.l, r1, stride), rhs_norm(a.f, s.l, r1, stride), stride, i);
          dot_acc(red0, f0, o0);
          dot_acc(red1, f1, o1);
        } else if (EPI == EPI_OMEGA) {
          pair_split(xv, f0, f1);
          dot_acc(red0, o0, f0);
          dot_acc(red1, o1, f1);
          red0[2] += norm_site(o0);
          red1[2] += norm_site(o1);
        } else {
          red0[0] += norm_site(o0);
          red1[0] += norm_site(o1);
        }
      }
    }
    c2 res[12];
    if (MODE & MODE_POST) {
      pair_hermitian6(res, crow, acc);
      pair_hermitian6(res + 6, crow + 72, acc + 6);
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) res[k] = acc[k];
    }
    cpx<float> y0[12], y1[12];
    pair_split(res, y0, y1);
    if (act0)
      SpinorIO<P>::template store<true>(y0, rhs_ptr_w<P>(a.out, s.l, r0, stride), rhs_norm(a.out, s.l, r0, stride),
                                        stride, i);
    if (act1)
      SpinorIO<P>::template store<true>(y1, rhs_ptr_w<P>(a.out, s.l, r1, stride), rhs_norm(a.out, s.l, r1, stride),
                                        stride, i);
  }
  if constexpr (EPI != EPI_NONE) {
    // the block is a whole number of warps and TS divides 32: the TS lanes of a pair
    // are one aligned group of a warp
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
      for (int o = TS / 2; o; o >>= 1) {
        red0[k] += __shfl_xor_sync(0xffffffffu, red0[k], o);
        red1[k] += __shfl_xor_sync(0xffffffffu, red1[k], o);
      }
    if (ls == 0) {
      if (act0) {
        double* dst = a.partials + ((size_t)(slot0 + r0) * a.maxch + s.chunk) * 3;
        dst[0] = red0[0];
        dst[1] = red0[1];
        dst[2] = red0[2];
      }
      if (act1) {
        double* dst = a.partials + ((size_t)(slot0 + r1) * a.maxch + s.chunk) * 3;
        dst[0] = red1[0];
        dst[1] = red1[1];
        dst[2] = red1[2];
      }
    }
  }
}

// dynamic shared memory of the pair kernel with TS sites per CTA
inline size_t pair_smem_bytes(int ts) { return (size_t)(8 * PAIR_LROW + PAIR_CROW) * ts * sizeof(float); }

template <int P>
cudaError_t launch_dslash_pair(const DslashArgs& a, bool dagger, int mode, int ts, cudaStream_t st);

#define WCL_PAIR_CASE(P, DAG, MODE, EPI)                                                                   \
  case (MODE) | ((DAG) ? 16 : 0) | ((EPI) << 5): {                                                        \
    const size_t sm = pair_smem_bytes(ts);                                                                \
    cudaError_t ea;                                                                                       \
    if (ts == 32) {                                                                                       \
      ea = allow_dynamic_smem(dslash_pair_kernel<P, DAG, MODE, EPI, 32>, sm);                            \
      if (ea != cudaSuccess) return ea;                                                                   \
      dslash_pair_kernel<P, DAG, MODE, EPI, 32><<<a.b.total_blocks, threads, sm, st>>>(a);              \
    } else if (ts == 8) {                                                                                 \
      dslash_pair_kernel<P, DAG, MODE, EPI, 8><<<a.b.total_blocks, threads, sm, st>>>(a);               \
    } else {                                                                                              \
      dslash_pair_kernel<P, DAG, MODE, EPI, 16><<<a.b.total_blocks, threads, sm, st>>>(a);              \
    }                                                                                                     \
    fin = EPI;                                                                                            \
    break;                                                                                                \
  }

// ts: sites per CTA (8, 16 or 32); the geometry a.b must have been built with that tile
#define WCL_DEFINE_PAIR_LAUNCHER(P)                                                                        \
  template <>                                                                                             \
  cudaError_t launch_dslash_pair<P>(const DslashArgs& a, bool dagger, int mode, int ts, cudaStream_t st) { \
    if (ts != 8 && ts != 16 && ts != 32) return cudaErrorInvalidValue;                                    \
    const int npair = (a.nrhs_tc + 1) / 2;                                                                 \
    const int threads = (ts * npair + 31) / 32 * 32;                                                       \
    if (threads > (ts == 32 ? 256 : ts == 16 ? 128 : 64)) return cudaErrorInvalidValue;                   \
    int fin = 0;                                                                                           \
    switch (mode | (dagger ? 16 : 0)) {                                                                    \
      WCL_PAIR_CASE(P, false, MODE_POST, EPI_NONE)                                                         \
      WCL_PAIR_CASE(P, true, MODE_POST, EPI_NONE)                                                          \
      WCL_PAIR_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_NONE)                                              \
      WCL_PAIR_CASE(P, true, MODE_XPAY | MODE_PRE, EPI_NONE)                                               \
      WCL_PAIR_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_ALPHA)                                             \
      WCL_PAIR_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_OMEGA)                                             \
      WCL_PAIR_CASE(P, false, MODE_XPAY | MODE_PRE, EPI_CGALPHA)                                           \
      WCL_PAIR_CASE(P, true, MODE_XPAY | MODE_PRE, EPI_CGZ)                                                \
      default: return cudaErrorInvalidValue;                                                               \
    }                                                                                                      \
    cudaError_t e = cudaGetLastError();                                                                    \
    if (e != cudaSuccess) return e;                                                                        \
    return launch_epi_finalize(fin, a, st);                                                                \
  }

}  // namespace wcl
