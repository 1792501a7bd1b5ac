// Multi-RHS fused dslash + clover on the tensor cores, 16-bit storage.
//
// With many right-hand sides the link multiply of the hopping term is a dense
// contraction: for one site and one direction mu,
//   Y[rhs][(colour', re/im)] = sum_k H[rhs][k] B[k][(colour', re/im)],
// where H holds the projected half spinors of every RHS and B is the real
// form of the link.  Each warp owns one site at a time and all its RHS (up to
// 16 MMA rows).  Per direction mu the forward hop (U_mu(x), colour index
// k = 0..5) and the backward hop (U_mu(x-mu)^+, k = 8..13) are stacked in K,
// so one mma.sync.m16n8k16 (f16 inputs, FP32 accumulation) per output spin
// adds both hops; the spin reconstruction (rows 2, 3 = +-h or +-i h) is folded
// into the A operand.  The clover term is a second contraction over
// (spin, colour) of a chiral block, fed directly from the FP32 accumulator
// fragments (whose layout is that of an f16 A fragment).
//
// Scaling: spinors are stored as value / per-(site, rhs) norm.  Before the
// MMAs every neighbour contribution of an RHS is rescaled to the largest norm
// among its 8 neighbours, so all A values are bounded by 2; the result is
// multiplied back by that norm.  Links are unit-bounded; clover blocks are
// stored divided by a per-site scale that multiplies the result.
//
// Fragment conventions (PTX m16n8k16, g = lane / 4, t = lane % 4):
//   A rows g, g+8 = rhs g, g+8;  A cols 2t, 2t+1 = colour t (re, im) of the
//   forward hop, cols 8+2t, 9+2t = colour t of the backward hop (t = 3: zero);
//   B col g = (colour g/2, re/im g%2) of the output (g >= 6: zero);
//   C row g / g+8, cols 2t, 2t+1 = output colour t (re, im).
#include "dslash.cuh"

namespace wcl {

constexpr int TC_WARPS = 4, TC_SPW = 4, TC_TILE = TC_WARPS * TC_SPW;  // sites per CTA
constexpr int TC_HSTRIDE = 12;  // half2 words per (dir, rhs) row of projected spinors (bank-conflict free)
constexpr int TC_XSTRIDE = 20;  // half2 words per rhs row of staged spinors at the site

struct TcWarpSmem {
  uint32_t h[8][16][TC_HSTRIDE];  // projected half spinors: word k*4 + colour, k = h0 / h1
  uint32_t link[8][9];            // eta * U (fwd) or eta * U (bwd, adjoint taken at use) as half2
  uint32_t clov[36];              // packed clover block pair (72 halves)
  uint32_t x[16][TC_XSTRIDE];     // spinor x at the site (word spin*4 + colour), XPAY
  uint32_t f[16][TC_XSTRIDE];     // rhat at the site, EPI_ALPHA
  uint32_t out[16][12];           // output staging, word 3*spin + colour
  float rowscale[16];             // largest neighbour norm per rhs
  float xnorm[16], fnorm[16], onorm[16];
  float red[16][3];               // epilogue partial sums per rhs
};

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ __half2 u2h(uint32_t w) { return *reinterpret_cast<__half2*>(&w); }
__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
// i * z for z = (re, im) in a half2
__device__ __forceinline__ __half2 hmul_i(__half2 z) {
  return __hmul2(__lowhigh2highlow(z), __halves2half2(__float2half(-1.f), __float2half(1.f)));
}
__device__ __forceinline__ __half2 hscale(__half2 z, float s) { return __hmul2(z, __float2half2_rn(s)); }
// c * z with c in {+1, -1, +i, -i}: code 0: +1, 1: -1, 2: +i, 3: -i
__device__ __forceinline__ __half2 hphase(__half2 z, int code) {
  if (code == 0) return z;
  if (code == 1) return __hneg2(z);
  if (code == 2) return hmul_i(z);
  return __hneg2(hmul_i(z));
}

// projector (1 + S gamma_mu) applied to the 4 spins p[0..3] of one colour -> h0, h1
template <int MU>
__device__ __forceinline__ void tc_project(const __half2 p[4], int S, __half2& h0, __half2& h1) {
  const __half2 p0 = p[0], p1 = p[1], p2 = p[2], p3 = p[3];
  if (MU == 0) {  // h0 = p0 + S i p3, h1 = p1 + S i p2
    h0 = (S > 0) ? __hadd2(p0, hmul_i(p3)) : __hsub2(p0, hmul_i(p3));
    h1 = (S > 0) ? __hadd2(p1, hmul_i(p2)) : __hsub2(p1, hmul_i(p2));
  } else if (MU == 1) {  // h0 = p0 - S p3, h1 = p1 + S p2
    h0 = (S > 0) ? __hsub2(p0, p3) : __hadd2(p0, p3);
    h1 = (S > 0) ? __hadd2(p1, p2) : __hsub2(p1, p2);
  } else if (MU == 2) {  // h0 = p0 + S i p2, h1 = p1 - S i p3
    h0 = (S > 0) ? __hadd2(p0, hmul_i(p2)) : __hsub2(p0, hmul_i(p2));
    h1 = (S > 0) ? __hsub2(p1, hmul_i(p3)) : __hadd2(p1, hmul_i(p3));
  } else {  // h0 = p0 + S p2, h1 = p1 + S p3
    h0 = (S > 0) ? __hadd2(p0, p2) : __hsub2(p0, p2);
    h1 = (S > 0) ? __hadd2(p1, p3) : __hsub2(p1, p3);
  }
}

// reconstruction of output spin sp (0..3) from (h0, h1) of direction MU with sign S:
// returns which component (0: h0, 1: h1) and the phase code
template <int MU>
__device__ __forceinline__ void tc_recon(int sp, int S, int& comp, int& code) {
  if (sp < 2) {
    comp = sp;
    code = 0;
    return;
  }
  // rows 2, 3 for (1 + S gamma): mu=x: -S i h1, -S i h0; mu=y: S h1, -S h0;
  //                             mu=z: -S i h0,  S i h1; mu=t: S h0,   S h1
  int c_plus_one = 0, c_i = 0;  // sign (+1 => 0, -1 => 1) and whether an i factor appears
  if (MU == 0) {
    comp = (sp == 2) ? 1 : 0;
    c_i = 1;
    c_plus_one = (S > 0) ? 1 : 0;  // -S
  } else if (MU == 1) {
    comp = (sp == 2) ? 1 : 0;
    c_i = 0;
    c_plus_one = (sp == 2) ? ((S > 0) ? 0 : 1) : ((S > 0) ? 1 : 0);
  } else if (MU == 2) {
    comp = (sp == 2) ? 0 : 1;
    c_i = 1;
    c_plus_one = (sp == 2) ? ((S > 0) ? 1 : 0) : ((S > 0) ? 0 : 1);
  } else {
    comp = (sp == 2) ? 0 : 1;
    c_i = 0;
    c_plus_one = (S > 0) ? 0 : 1;
  }
  code = c_i ? (2 + c_plus_one) : c_plus_one;
}

// clover B-fragment lookup for this lane: block b, output spin j (local), input spin si (local)
struct ClovIdx {
  uint8_t word;   // half2 word of the packed pair (re, im) or diagonal half
  uint8_t kind;   // 0: zero, 1: diagonal (real), 2: lower (as stored), 3: upper (conjugate of lower)
  uint8_t hi;     // diagonal: which half of the word
};

__device__ __forceinline__ ClovIdx clov_index(int b, int row, int col) {
  ClovIdx c;
  c.hi = 0;
  if (row == col) {
    const int half_index = 36 * b + row;  // diagonal halves 0..5 of block b
    c.word = (uint8_t)(half_index >> 1);
    c.hi = (uint8_t)(half_index & 1);
    c.kind = 1;
  } else {
    const int r = row > col ? row : col, cc = row > col ? col : row;
    const int k = r * (r - 1) / 2 + cc;
    c.word = (uint8_t)((36 * b + 6 + 2 * k) >> 1);
    c.kind = row > col ? 2 : 3;
  }
  return c;
}

// real-form B pair (b0, b1) for complex entry z at output re/im index reim:
// reim 0: (Re z, -Im z); reim 1: (Im z, Re z)
__device__ __forceinline__ uint32_t bpair(__half2 z, int reim) {
  const __half re = __low2half(z), im = __high2half(z);
  return reim == 0 ? h2u(__halves2half2(re, __hneg(im))) : h2u(__halves2half2(im, re));
}

__device__ __forceinline__ __half2 clov_entry(const uint32_t* clov, ClovIdx c) {
  if (c.kind == 0) return __float2half2_rn(0.f);
  const __half2 w = u2h(clov[c.word]);
  if (c.kind == 1) return __halves2half2(c.hi ? __high2half(w) : __low2half(w), __float2half(0.f));
  if (c.kind == 2) return w;
  return __halves2half2(__low2half(w), __hneg(__high2half(w)));
}

template <int P, bool DAG, int MODE, int EPI>
__global__ void __launch_bounds__(TC_WARPS * 32) dslash_tc_kernel(const __grid_constant__ DslashArgs a) {
  __shared__ TcWarpSmem smem_all[TC_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  TcWarpSmem& sm = smem_all[warp];
  const int g = lane >> 2, t = lane & 3;
  const Slice s = find_slice(a.b, blockIdx.x);  // geometry with one slice per lattice
  const LatGeom& G = a.b.lat[s.l];
  const int nrhs = a.nrhs_tc;
  const long stride = G.stride;
  const int p = a.out_parity;
  constexpr int SF = DAG ? +1 : -1, SB = -SF;
  const int slot0 = s.l * nrhs;

  // per-lane clover fragment lookups (block b, output spin j) -> (s_in 0, s_in 1)
  ClovIdx cl[2][2][2];
#pragma unroll
  for (int b = 0; b < 2; b++)
#pragma unroll
    for (int j = 0; j < 2; j++)
#pragma unroll
      for (int si = 0; si < 2; si++) {
        if (t < 3 && g < 6)
          cl[b][j][si] = clov_index(b, 3 * j + g / 2, 3 * si + t);
        else
          cl[b][j][si].kind = 0, cl[b][j][si].word = 0, cl[b][j][si].hi = 0;
      }

  // rows this lane stages: rhs r = lane & 15, side = lane >> 4 (0 forward, 1 backward hops)
  const int sr = lane & 15, side = lane >> 4;
  const bool r_ok = sr < nrhs && (!a.active || a.active[slot0 + sr]);
  const void* in_r = r_ok ? rhs_ptr<P>(a.in, s.l, sr, stride) : nullptr;
  const float* in_n = r_ok ? rhs_norm(a.in, s.l, sr, stride) : nullptr;

  float red_acc[2][3] = {{0, 0, 0}, {0, 0, 0}};  // rows g, g+8

  const long site0 = (long)s.chunk * TC_TILE + warp * TC_SPW;
  for (int ks = 0; ks < TC_SPW; ks++) {
    const long i = site0 + ks;
    if (i >= G.vh) break;
    // neighbour indices (every lane computes the same)
    const int lxh = G.lxh, Lx = G.dims[0], Ly = G.dims[1], Lz = G.dims[2], Lt = G.dims[3];
    const int xh = (int)(i % lxh);
    int rem = (int)(i / lxh);
    const int y = rem % Ly;
    rem /= Ly;
    const int z = rem % Lz;
    const int tt = rem / Lz;
    const int x = 2 * xh + ((p + y + z + tt) & 1);
    const long row = i - xh;
    const long plane = (long)lxh * Ly, vol3 = plane * Lz;
    long jn[8];
    jn[0] = row + ((x + 1 == Lx ? 0 : x + 1) >> 1);
    jn[1] = row + ((x == 0 ? Lx - 1 : x - 1) >> 1);
    jn[2] = (y + 1 == Ly) ? i - (long)(Ly - 1) * lxh : i + lxh;
    jn[3] = (y == 0) ? i + (long)(Ly - 1) * lxh : i - lxh;
    jn[4] = (z + 1 == Lz) ? i - (long)(Lz - 1) * plane : i + plane;
    jn[5] = (z == 0) ? i + (long)(Lz - 1) * plane : i - plane;
    jn[6] = (tt + 1 == Lt) ? i - (long)(Lt - 1) * vol3 : i + vol3;
    jn[7] = (tt == 0) ? i + (long)(Lt - 1) * vol3 : i - vol3;
    const float eta_f = (tt + 1 == Lt) ? G.tbw_f : G.tw_f, eta_b = (tt == 0) ? G.tbw_f : G.tw_f;

    // ---- stage norms and the row scale (largest neighbour norm of each rhs) ----
    float nrm[4];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) nrm[mu] = r_ok ? __ldg(in_n + jn[2 * mu + side]) : 0.f;
    float mx = fmaxf(fmaxf(nrm[0], nrm[1]), fmaxf(nrm[2], nrm[3]));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
    const float inv_mx = mx > 0.f ? 1.f / mx : 0.f;
    if (side == 0) sm.rowscale[sr] = mx;

    // ---- stage projected half spinors of the 4 directions of this side ----
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      uint32_t* hdst = sm.h[2 * mu + side][sr];
      if (r_ok) {
        const uint4* src = static_cast<const uint4*>(in_r);
        const long j = jn[2 * mu + side];
        const uint4 q0 = ldg(src + j), q1 = ldg(src + stride + j), q2 = ldg(src + 2 * stride + j);
        const uint32_t w[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
        const float f = nrm[mu] * inv_mx;
        const int S = side ? SB : SF;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const __half2 pp[4] = {u2h(w[c]), u2h(w[3 + c]), u2h(w[6 + c]), u2h(w[9 + c])};
          __half2 h0, h1;
          if (mu == 0) tc_project<0>(pp, S, h0, h1);
          else if (mu == 1) tc_project<1>(pp, S, h0, h1);
          else if (mu == 2) tc_project<2>(pp, S, h0, h1);
          else tc_project<3>(pp, S, h0, h1);
          hdst[c] = h2u(hscale(h0, f));
          hdst[4 + c] = h2u(hscale(h1, f));
        }
      } else {
#pragma unroll
        for (int c = 0; c < 3; c++) hdst[c] = hdst[4 + c] = 0u;
      }
    }
    // ---- stage links (lanes 0..7: direction d) and the clover (lanes 8..16) ----
    if (lane < 8) {
      const int d = lane, mu = d >> 1;
      cpx<float> u[3][3];
      if (d & 1)
        LinkIO<P>::load(u, a.gauge[s.l][1 - p], stride, jn[d], mu);
      else
        LinkIO<P>::load(u, a.gauge[s.l][p], stride, i, mu);
      const float eta = (mu == 3) ? ((d & 1) ? eta_b : eta_f) : 1.f;
#pragma unroll
      for (int r2 = 0; r2 < 3; r2++)
#pragma unroll
        for (int c = 0; c < 3; c++) sm.link[d][3 * r2 + c] = h2u(__floats2half2_rn(eta * u[r2][c].re, eta * u[r2][c].im));
    } else if (lane < 17) {
      const void* cptr = (MODE & MODE_POST) ? a.cpost[s.l] : a.cpre[s.l];
      const uint4 q = ldg(static_cast<const uint4*>(cptr) + (long)(lane - 8) * stride + i);
      sm.clov[4 * (lane - 8) + 0] = q.x;
      sm.clov[4 * (lane - 8) + 1] = q.y;
      sm.clov[4 * (lane - 8) + 2] = q.z;
      sm.clov[4 * (lane - 8) + 3] = q.w;
    }
    const float cnorm = __ldg(((MODE & MODE_POST) ? a.cpost_norm[s.l] : a.cpre_norm[s.l]) + i);
    // x (and rhat) at the site for XPAY: lanes stage rhs sr (side 0: x, side 1: rhat)
    if (MODE & MODE_XPAY) {
      const bool want = (side == 0) || (EPI == EPI_ALPHA);
      if (want) {
        const FieldRef& F = side == 0 ? a.x : a.f;
        uint32_t* dst = side == 0 ? sm.x[sr] : sm.f[sr];
        if (r_ok) {
          const uint4* src = static_cast<const uint4*>(rhs_ptr<P>(F, s.l, sr, stride));
          const uint4 q0 = ldg(src + i), q1 = ldg(src + stride + i), q2 = ldg(src + 2 * stride + i);
          const uint32_t w[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
#pragma unroll
          for (int sp = 0; sp < 4; sp++)
#pragma unroll
            for (int c = 0; c < 3; c++) dst[sp * 4 + c] = w[3 * sp + c];
          const float nn = __ldg(rhs_norm(F, s.l, sr, stride) + i);
          if (side == 0) sm.xnorm[sr] = nn; else sm.fnorm[sr] = nn;
        } else {
#pragma unroll
          for (int k = 0; k < 16; k++) dst[k] = 0u;
          if (side == 0) sm.xnorm[sr] = 0.f; else sm.fnorm[sr] = 0.f;
        }
      }
    }
    __syncwarp();

    // ---- hopping term: per mu, 4 MMAs (one per output spin) ----
    float acc[4][4];
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
      for (int k = 0; k < 4; k++) acc[sp][k] = 0.f;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      // B: rows 2t,2t+1 = forward colour t, rows 2t+8, 2t+9 = backward colour t; col g
      uint32_t bb[2] = {0u, 0u};
      if (t < 3 && g < 6) {
        const int cp = g >> 1, reim = g & 1;
        bb[0] = bpair(u2h(sm.link[2 * mu][3 * cp + t]), reim);  // U_f[cp][t]
        const __half2 ub = u2h(sm.link[2 * mu + 1][3 * t + cp]);  // U_b[t][cp]; (U_b^+)[cp][t] = conj
        bb[1] = bpair(__halves2half2(__low2half(ub), __hneg(__high2half(ub))), reim);
      }
      // A values: h_f, h_b for rows g, g+8, colour t (zero for t = 3)
      __half2 hf[2][2], hb[2][2];  // [row][comp]
#pragma unroll
      for (int rr = 0; rr < 2; rr++)
#pragma unroll
        for (int k = 0; k < 2; k++) {
          if (t < 3) {
            hf[rr][k] = u2h(sm.h[2 * mu][g + 8 * rr][4 * k + t]);
            hb[rr][k] = u2h(sm.h[2 * mu + 1][g + 8 * rr][4 * k + t]);
          } else {
            hf[rr][k] = hb[rr][k] = __float2half2_rn(0.f);
          }
        }
#pragma unroll
      for (int sp = 0; sp < 4; sp++) {
        int cf, codef, cb, codeb;
        if (mu == 0) { tc_recon<0>(sp, SF, cf, codef); tc_recon<0>(sp, SB, cb, codeb); }
        else if (mu == 1) { tc_recon<1>(sp, SF, cf, codef); tc_recon<1>(sp, SB, cb, codeb); }
        else if (mu == 2) { tc_recon<2>(sp, SF, cf, codef); tc_recon<2>(sp, SB, cb, codeb); }
        else { tc_recon<3>(sp, SF, cf, codef); tc_recon<3>(sp, SB, cb, codeb); }
        uint32_t aa[4];
        aa[0] = h2u(hphase(hf[0][cf], codef));
        aa[1] = h2u(hphase(hf[1][cf], codef));
        aa[2] = h2u(hphase(hb[0][cb], codeb));
        aa[3] = h2u(hphase(hb[1][cb], codeb));
        mma16816(acc[sp], aa, bb);
      }
    }

    // ---- clover and the combination ----
    float res[4][4];
    const float rs0 = sm.rowscale[g], rs1 = sm.rowscale[g + 8];
    const float alpha = (float)a.alpha[s.l];
    if (MODE & MODE_POST) {
      // out = A^-1 (alpha * rowscale * acc): clover MMA on the accumulators
#pragma unroll
      for (int b = 0; b < 2; b++) {
        uint32_t aa[4];
        aa[0] = h2u(__floats2half2_rn(acc[2 * b][0], acc[2 * b][1]));
        aa[1] = h2u(__floats2half2_rn(acc[2 * b][2], acc[2 * b][3]));
        aa[2] = h2u(__floats2half2_rn(acc[2 * b + 1][0], acc[2 * b + 1][1]));
        aa[3] = h2u(__floats2half2_rn(acc[2 * b + 1][2], acc[2 * b + 1][3]));
#pragma unroll
        for (int j = 0; j < 2; j++) {
          uint32_t bb[2] = {0u, 0u};
          if (t < 3 && g < 6) {
            bb[0] = bpair(clov_entry(sm.clov, cl[b][j][0]), g & 1);
            bb[1] = bpair(clov_entry(sm.clov, cl[b][j][1]), g & 1);
          }
          float c4[4] = {0.f, 0.f, 0.f, 0.f};
          mma16816(c4, aa, bb);
          const float s0 = alpha * rs0 * cnorm, s1 = alpha * rs1 * cnorm;
          res[2 * b + j][0] = s0 * c4[0];
          res[2 * b + j][1] = s0 * c4[1];
          res[2 * b + j][2] = s1 * c4[2];
          res[2 * b + j][3] = s1 * c4[3];
        }
      }
    } else {
      // out = alpha * rowscale * acc + beta * A x
      const float beta = (float)a.beta[s.l];
      const float xn0 = sm.xnorm[g], xn1 = sm.xnorm[g + 8];
#pragma unroll
      for (int b = 0; b < 2; b++) {
        uint32_t aa[4];
        aa[0] = t < 3 ? sm.x[g][(2 * b) * 4 + t] : 0u;
        aa[1] = t < 3 ? sm.x[g + 8][(2 * b) * 4 + t] : 0u;
        aa[2] = t < 3 ? sm.x[g][(2 * b + 1) * 4 + t] : 0u;
        aa[3] = t < 3 ? sm.x[g + 8][(2 * b + 1) * 4 + t] : 0u;
#pragma unroll
        for (int j = 0; j < 2; j++) {
          uint32_t bb[2] = {0u, 0u};
          if (t < 3 && g < 6) {
            bb[0] = bpair(clov_entry(sm.clov, cl[b][j][0]), g & 1);
            bb[1] = bpair(clov_entry(sm.clov, cl[b][j][1]), g & 1);
          }
          float c4[4] = {0.f, 0.f, 0.f, 0.f};
          mma16816(c4, aa, bb);
          const int sp = 2 * b + j;
          res[sp][0] = alpha * rs0 * acc[sp][0] + beta * xn0 * cnorm * c4[0];
          res[sp][1] = alpha * rs0 * acc[sp][1] + beta * xn0 * cnorm * c4[1];
          res[sp][2] = alpha * rs1 * acc[sp][2] + beta * xn1 * cnorm * c4[2];
          res[sp][3] = alpha * rs1 * acc[sp][3] + beta * xn1 * cnorm * c4[3];
        }
      }
      if (EPI != EPI_NONE && t < 3) {
        // per-lane contributions to the fused reductions (rows g, g+8)
#pragma unroll
        for (int rr = 0; rr < 2; rr++) {
#pragma unroll
          for (int sp = 0; sp < 4; sp++) {
            const float yr = res[sp][2 * rr], yi = res[sp][2 * rr + 1];
            if (EPI == EPI_ALPHA) {
              const float fnrm = sm.fnorm[g + 8 * rr];
              const float2 fv = __half22float2(u2h(sm.f[g + 8 * rr][sp * 4 + t]));
              const float fr = fv.x * fnrm, fi = fv.y * fnrm;
              red_acc[rr][0] += fr * yr + fi * yi;  // <f, y>
              red_acc[rr][1] += fr * yi - fi * yr;
            } else if (EPI == EPI_OMEGA) {
              const float xnrm = sm.xnorm[g + 8 * rr];
              const float2 xv = __half22float2(u2h(sm.x[g + 8 * rr][sp * 4 + t]));
              const float xr = xv.x * xnrm, xi = xv.y * xnrm;
              red_acc[rr][0] += yr * xr + yi * xi;  // <y, x>
              red_acc[rr][1] += yr * xi - yi * xr;
              red_acc[rr][2] += yr * yr + yi * yi;
            } else {
              red_acc[rr][0] += yr * yr + yi * yi;
            }
          }
        }
      }
    }

    // ---- store: per-rhs norm (max over 24 reals), f16 values via the staging rows ----
    float m0 = 0.f, m1 = 0.f;
    if (t < 3) {
#pragma unroll
      for (int sp = 0; sp < 4; sp++) {
        m0 = fmaxf(m0, fmaxf(fabsf(res[sp][0]), fabsf(res[sp][1])));
        m1 = fmaxf(m1, fmaxf(fabsf(res[sp][2]), fabsf(res[sp][3])));
      }
    }
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 1));
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, 2));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 1));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, 2));
    const float i0 = m0 > 0.f ? 1.f / m0 : 0.f, i1 = m1 > 0.f ? 1.f / m1 : 0.f;
    if (t < 3) {
#pragma unroll
      for (int sp = 0; sp < 4; sp++) {
        sm.out[g][3 * sp + t] = pack2<P>(res[sp][0] * i0, res[sp][1] * i0);
        sm.out[g + 8][3 * sp + t] = pack2<P>(res[sp][2] * i1, res[sp][3] * i1);
      }
    }
    if (t == 0) {
      sm.onorm[g] = m0;
      sm.onorm[g + 8] = m1;
    }
    __syncwarp();
    // 3 chunks per rhs: lane handles (rhs, chunk) pairs
    for (int e = lane; e < 3 * nrhs; e += 32) {
      const int r = e / 3, k = e % 3;
      if (a.active && !a.active[slot0 + r]) continue;
      uint4 q;
      q.x = sm.out[r][4 * k + 0];
      q.y = sm.out[r][4 * k + 1];
      q.z = sm.out[r][4 * k + 2];
      q.w = sm.out[r][4 * k + 3];
      uint4* dst = static_cast<uint4*>(rhs_ptr_w<P>(a.out, s.l, r, stride));
      dst[(long)k * stride + i] = q;
      if (k == 0) rhs_norm(a.out, s.l, r, stride)[i] = sm.onorm[r];
    }
    __syncwarp();
  }

  if (EPI != EPI_NONE) {
    // reduce the rows over the quad, then over the warps of the CTA; one partial per (CTA, rhs)
#pragma unroll
    for (int rr = 0; rr < 2; rr++)
#pragma unroll
      for (int k = 0; k < 3; k++) {
        float v = red_acc[rr][k];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        red_acc[rr][k] = v;
      }
    if (t == 0) {
#pragma unroll
      for (int k = 0; k < 3; k++) {
        sm.red[g][k] = red_acc[0][k];
        sm.red[g + 8][k] = red_acc[1][k];
      }
    }
    __syncthreads();
    if (threadIdx.x < nrhs) {
      const int r = threadIdx.x;
      double tot[3] = {0, 0, 0};
      for (int w = 0; w < TC_WARPS; w++)
        for (int k = 0; k < 3; k++) tot[k] += (double)smem_all[w].red[r][k];
      double* dst = a.partials + ((size_t)(slot0 + r) * a.maxch + s.chunk) * 3;
      dst[0] = tot[0];
      dst[1] = tot[1];
      dst[2] = tot[2];
    }
  }
}

#define WCL_TC_CASE(DAG, MODE, EPI)                                                        \
  case (MODE) | ((DAG) ? 16 : 0) | ((EPI) << 5):                                          \
    dslash_tc_kernel<P, DAG, MODE, EPI><<<a.b.total_blocks, TC_WARPS * 32, 0, st>>>(a);   \
    fin = EPI;                                                                            \
    break;

template <int P>
cudaError_t launch_dslash_tc_p(const DslashArgs& a, bool dagger, int mode, cudaStream_t st) {
  int fin = 0;
  switch (mode | (dagger ? 16 : 0)) {
    WCL_TC_CASE(false, MODE_POST, EPI_NONE)
    WCL_TC_CASE(true, MODE_POST, EPI_NONE)
    WCL_TC_CASE(false, MODE_XPAY | MODE_PRE, EPI_NONE)
    WCL_TC_CASE(true, MODE_XPAY | MODE_PRE, EPI_NONE)
    WCL_TC_CASE(false, MODE_XPAY | MODE_PRE, EPI_ALPHA)
    WCL_TC_CASE(false, MODE_XPAY | MODE_PRE, EPI_OMEGA)
    WCL_TC_CASE(false, MODE_XPAY | MODE_PRE, EPI_CGALPHA)
    WCL_TC_CASE(true, MODE_XPAY | MODE_PRE, EPI_CGZ)
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_epi_finalize(fin, a, st);
}

cudaError_t launch_dslash_tc(int prec, const DslashArgs& a, bool dagger, int mode, cudaStream_t st) {
  if (prec == F16) return launch_dslash_tc_p<F16>(a, dagger, mode, st);
  return cudaErrorInvalidValue;
}

int tc_tile_sites() { return TC_TILE; }

}  // namespace wcl
