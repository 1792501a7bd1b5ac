// PTC network layer and weight-gradient kernels (see ptc.cuh).
#include "ptc.cuh"

namespace wcl {

// T_s psi at output site i of parity p (input on parity 1-p for s != 0).
// s = 0: identity; s = 1 + 2 mu: +mu; s = 2 + 2 mu: -mu.
struct Nbr {
  long jf[4], jb[4];
  float sf, sb;  // time-boundary signs of the t hops
};

__device__ __forceinline__ Nbr neighbours(const LatGeom& g, int p, long i) {
  Nbr n;
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
  n.sf = (t + 1 == Lt) ? g.tb : 1.f;
  n.sb = (t == 0) ? g.tb : 1.f;
  return n;
}

__device__ __forceinline__ void transport(cpx<float> out[12], int s, const float4* f_here, const float4* f_there,
                                          const void* g_here, const void* g_there, long stride, long i,
                                          const Nbr& n) {
  if (s == 0) {
    SpinorIO<F32>::load(out, f_here, nullptr, stride, i);
    return;
  }
  const int mu = (s - 1) >> 1;
  const bool back = ((s - 1) & 1) != 0;
  cpx<float> psi[12], u[3][3];
  if (!back) {
    SpinorIO<F32>::load(psi, f_there, nullptr, stride, n.jf[mu]);
    LinkIO<F32>::load(u, g_here, stride, i, mu);
    const float sg = (mu == 3) ? n.sf : 1.f;
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
      for (int a = 0; a < 3; a++) {
        cpx<float> acc = {0, 0};
#pragma unroll
        for (int b = 0; b < 3; b++) cfma(acc, u[a][b], psi[3 * sp + b]);
        out[3 * sp + a] = sg * acc;
      }
  } else {
    SpinorIO<F32>::load(psi, f_there, nullptr, stride, n.jb[mu]);
    LinkIO<F32>::load(u, g_there, stride, n.jb[mu], mu);
    const float sg = (mu == 3) ? n.sb : 1.f;
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
      for (int a = 0; a < 3; a++) {
        cpx<float> acc = {0, 0};
#pragma unroll
        for (int b = 0; b < 3; b++) cfma_conj(acc, u[b][a], psi[3 * sp + b]);
        out[3 * sp + a] = sg * acc;
      }
  }
}

// One layer, four lanes per output site: lane q transports input channel q (if
// q < cin) along each shift and accumulates output channel q (if q < cout); the
// four transported spinors of a shift are exchanged by warp shuffles, so each
// transport is computed once and a thread holds one accumulator, not four.
// Weights live in shared memory with the output-channel stride padded by one
// complex so that the four lanes' reads fall in different banks.
constexpr int PTC_SITES_PER_CTA = 32;  // 128 threads
constexpr int PTC_WSTRIDE = PTC_MAXC * PTC_NSHIFT * 16 + 1;

__global__ void __launch_bounds__(128) ptc_layer_kernel(const __grid_constant__ PtcLayerArgs a) {
  __shared__ float2 w_s[PTC_MAXC * PTC_WSTRIDE];
  const int per_co = a.cin * PTC_NSHIFT * 16;
  for (int k = threadIdx.x; k < a.cout * per_co; k += blockDim.x) {
    const int co = k / per_co, r = k - co * per_co;
    w_s[co * PTC_WSTRIDE + r] = a.use_bf16 ? __bfloat1622float2(a.wb[k]) : a.w[k];
  }
  __syncthreads();
  const Slice s = find_slice(a.b, blockIdx.x);
  const LatGeom& g = a.b.lat[s.l];
  const int q = threadIdx.x & 3;
  const long i = (long)s.chunk * PTC_SITES_PER_CTA + (threadIdx.x >> 2);
  const bool site_ok = i < g.vh;  // lanes past the end still take part in the shuffles
  const long ii = site_ok ? i : 0;
  const long stride = g.stride;
  const int p = a.parity;
  const Nbr n = neighbours(g, p, ii);
  const void* g_here = a.gauge[s.l][p];
  const void* g_there = a.gauge[s.l][1 - p];
  const int qin = q < a.cin ? q : 0;
  const float4* f_here = a.in[s.l] + ptc_field_offset(s.rhs, qin, a.cin, p, stride);
  const float4* f_there = a.in[s.l] + ptc_field_offset(s.rhs, qin, a.cin, 1 - p, stride);
  const float2* wq = w_s + (q < a.cout ? q : 0) * PTC_WSTRIDE;
  const int lane0 = (threadIdx.x & 31) & ~3;

  cpx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = {0.f, 0.f};

#pragma unroll 1
  for (int sh = 0; sh < PTC_NSHIFT; sh++) {
    cpx<float> t[12];
    if (q < a.cin) {
      transport(t, sh, f_here, f_there, g_here, g_there, stride, ii, n);
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) t[k] = {0.f, 0.f};
    }
#pragma unroll 1
    for (int ci = 0; ci < a.cin; ci++) {
      cpx<float> u[12];
#pragma unroll
      for (int k = 0; k < 12; k++) {
        u[k].re = __shfl_sync(0xffffffffu, t[k].re, lane0 + ci);
        u[k].im = __shfl_sync(0xffffffffu, t[k].im, lane0 + ci);
      }
      const float2* w = wq + (ci * PTC_NSHIFT + sh) * 16;
#pragma unroll
      for (int al = 0; al < 4; al++)
#pragma unroll
        for (int be = 0; be < 4; be++) {
          const float2 wv = w[al * 4 + be];
          const cpx<float> wc = {wv.x, wv.y};
#pragma unroll
          for (int col = 0; col < 3; col++) cfma(acc[3 * al + col], wc, u[3 * be + col]);
        }
    }
  }
  if (!site_ok || q >= a.cout) return;
  float4* o = a.out[s.l] + ptc_field_offset(s.rhs, q, a.cout, p, stride);
  if (a.accumulate) {
    cpx<float> prev[12];
    SpinorIO<F32>::load<false>(prev, o, nullptr, stride, i);
#pragma unroll
    for (int k = 0; k < 12; k++) acc[k] = acc[k] + prev[k];
  }
  SpinorIO<F32>::store(acc, o, nullptr, stride, i);
}

int ptc_layer_sites_per_cta() { return PTC_SITES_PER_CTA; }

// ---------------------------------------------------------------------------
// Tensor-core layer (BF16 weights): the channel and spin mixing of every shift s
// as a real GEMM on mma.sync.m16n8k16 (BF16 inputs, FP32 accumulation),
//   C[(co, alpha, re/im)][site] += A_s[(co, alpha, re/im)][(ci, beta, re/im)] B_s[(ci, beta, re/im)][site],
// one GEMM per colour.  A_s holds W[co][ci][s] in real form [[Re, -Im], [Im, Re]]
// (exact: the weights are BF16).  B_s holds the transported inputs split into three
// BF16 terms (hi + mid + lo carry 24 significant bits), so the sum matches the FP32
// layer to FP32 rounding.  Lane (g, q) = (lane / 4, lane % 4): g is the site within
// the warp's 8 sites; q is the input channel the lane transports, the spin beta of
// the B values it holds and the output channel it stores.
//
// m16n8k16 fragments (g = lane / 4, t = lane % 4), k = ci_local * 8 + beta * 2 + re/im
// within a k-step, m = co * 8 + alpha * 2 + re/im:
//   A regs: (row g, k 2t..2t+1), (row g+8, k 2t..), (row g, k 2t+8..), (row g+8, k 2t+8..)
//   B regs: (k 2t..2t+1, col g), (k 2t+8..2t+9, col g)
//   C     : (row g, cols 2t, 2t+1), (row g+8, cols 2t, 2t+1)

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

// A fragments of one layer, [shift][mt][j][lane] (4 registers each)
__global__ void ptc_pack_frag_kernel(const __nv_bfloat162* __restrict__ wb, int cin, int cout, int MT, int J,
                                     uint4* __restrict__ frag) {
  const int n = PTC_NSHIFT * MT * J * 32;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int lane = e & 31, j = (e >> 5) % J, mt = (e / (32 * J)) % MT, sh = e / (32 * J * MT);
  const int g = lane >> 2, t = lane & 3;
  uint32_t r[4];
  for (int reg = 0; reg < 4; reg++) {
    const int row = 16 * mt + g + ((reg & 1) ? 8 : 0);
    const int k0 = 16 * j + 2 * t + ((reg & 2) ? 8 : 0);
    const int co = row >> 3, al = (row >> 1) & 3, ro = row & 1;
    const int ci = k0 >> 3, be = (k0 >> 1) & 3;  // k0 even: re/im in = 0, 1
    float lo = 0.f, hi = 0.f;
    if (co < cout && ci < cin) {
      const float2 w = __bfloat1622float2(wb[((co * cin + ci) * PTC_NSHIFT + sh) * 16 + al * 4 + be]);
      // real form: row re: (Re, -Im); row im: (Im, Re)
      lo = ro ? w.y : w.x;
      hi = ro ? w.x : -w.y;
    }
    r[reg] = bf16x2_bits(__floats2bfloat162_rn(lo, hi));
  }
  frag[e] = make_uint4(r[0], r[1], r[2], r[3]);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint4& a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// (re, im) -> three BF16 pairs whose sum is the FP32 pair to 24 bits
__device__ __forceinline__ void split3(float2 v, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat162 vh = __floats2bfloat162_rn(v.x, v.y);
  const float2 fh = __bfloat1622float2(vh);
  const float rx = v.x - fh.x, ry = v.y - fh.y;
  const __nv_bfloat162 vm = __floats2bfloat162_rn(rx, ry);
  const float2 fm = __bfloat1622float2(vm);
  const __nv_bfloat162 vl = __floats2bfloat162_rn(rx - fm.x, ry - fm.y);
  h = bf16x2_bits(vh);
  m = bf16x2_bits(vm);
  l = bf16x2_bits(vl);
}

constexpr int PTC_TROW = 4 * 12 + 1;  // staged complex per site (+1 against bank conflicts)

template <int MT, int J>
__global__ void __launch_bounds__(128) ptc_layer_tc_kernel(const __grid_constant__ PtcLayerArgs a,
                                                           const uint4* __restrict__ frag) {
  __shared__ uint4 a_s[PTC_NSHIFT * MT * J * 32];
  __shared__ float2 t_s[4][8][PTC_TROW];
  for (int k = threadIdx.x; k < PTC_NSHIFT * MT * J * 32; k += blockDim.x) a_s[k] = frag[k];
  __syncthreads();
  const Slice s = find_slice(a.b, blockIdx.x);
  const LatGeom& g = a.b.lat[s.l];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gs = lane >> 2, q = lane & 3;
  const long i = (long)s.chunk * PTC_SITES_PER_CTA + warp * 8 + gs;
  const bool site_ok = i < g.vh;  // lanes past the end still take part in the MMAs
  const long ii = site_ok ? i : 0;
  const long stride = g.stride;
  const int p = a.parity;
  const Nbr n = neighbours(g, p, ii);
  const void* g_here = a.gauge[s.l][p];
  const void* g_there = a.gauge[s.l][1 - p];
  const int qin = q < a.cin ? q : 0;
  const float4* f_here = a.in[s.l] + ptc_field_offset(s.rhs, qin, a.cin, p, stride);
  const float4* f_there = a.in[s.l] + ptc_field_offset(s.rhs, qin, a.cin, 1 - p, stride);
  float2* my = t_s[warp][gs];

  float acc[MT][3][4];
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int r = 0; r < 4; r++) acc[mt][c][r] = 0.f;

#pragma unroll 1
  for (int sh = 0; sh < PTC_NSHIFT; sh++) {
    cpx<float> t[12];
    if (q < a.cin) {
      transport(t, sh, f_here, f_there, g_here, g_there, stride, ii, n);
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) t[k] = {0.f, 0.f};
    }
#pragma unroll
    for (int k = 0; k < 12; k++) my[q * 12 + k] = make_float2(t[k].re, t[k].im);
    __syncwarp();
    float2 v[2 * J][3];  // spin q of input channels 0 .. 2J-1, three colours
#pragma unroll
    for (int ci = 0; ci < 2 * J; ci++)
#pragma unroll
      for (int c = 0; c < 3; c++) v[ci][c] = my[ci * 12 + q * 3 + c];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < J; j++) {
      uint4 af[MT];
#pragma unroll
      for (int mt = 0; mt < MT; mt++) af[mt] = a_s[((sh * MT + mt) * J + j) * 32 + lane];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        uint32_t h0, m0, l0, h1, m1, l1;
        split3(v[2 * j][c], h0, m0, l0);
        split3(v[2 * j + 1][c], h1, m1, l1);
#pragma unroll
        for (int mt = 0; mt < MT; mt++) {
          mma_bf16(acc[mt][c], af[mt], h0, h1);
          mma_bf16(acc[mt][c], af[mt], m0, m1);
          mma_bf16(acc[mt][c], af[mt], l0, l1);
        }
      }
    }
  }
  // epilogue: C fragments -> [site][co * 12 + alpha * 3 + colour] -> one output channel per lane
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int r = 0; r < 4; r++) {
        const int row = 16 * mt + gs + ((r & 2) ? 8 : 0);
        const int col = 2 * q + (r & 1);
        const int co = row >> 3, al = (row >> 1) & 3;
        float* dst = reinterpret_cast<float*>(&t_s[warp][col][co * 12 + al * 3 + c]);
        dst[row & 1] = acc[mt][c][r];
      }
  __syncwarp();
  if (!site_ok || q >= a.cout) return;
  cpx<float> o12[12];
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const float2 v2 = my[q * 12 + k];
    o12[k] = {v2.x, v2.y};
  }
  float4* o = a.out[s.l] + ptc_field_offset(s.rhs, q, a.cout, p, stride);
  if (a.accumulate) {
    cpx<float> prev[12];
    SpinorIO<F32>::load<false>(prev, o, nullptr, stride, i);
#pragma unroll
    for (int k = 0; k < 12; k++) o12[k] = o12[k] + prev[k];
  }
  SpinorIO<F32>::store(o12, o, nullptr, stride, i);
}

int ptc_frag_entries(int cin, int cout) {
  return PTC_NSHIFT * ((cout * 8 + 15) / 16) * ((cin * 8 + 15) / 16) * 32;
}

cudaError_t ptc_pack_frag(const __nv_bfloat162* wb, int cin, int cout, uint4* frag, cudaStream_t st) {
  const int MT = (cout * 8 + 15) / 16, J = (cin * 8 + 15) / 16;
  const int n = ptc_frag_entries(cin, cout);
  ptc_pack_frag_kernel<<<(n + 127) / 128, 128, 0, st>>>(wb, cin, cout, MT, J, frag);
  return cudaGetLastError();
}

cudaError_t ptc_layer(const PtcLayerArgs& a, cudaStream_t st, const uint4* frag) {
  if (a.cout < 1 || a.cout > PTC_MAXC || a.cin < 1 || a.cin > PTC_MAXC) return cudaErrorInvalidValue;
  if (frag && a.use_bf16) {
    const int MT = (a.cout * 8 + 15) / 16, J = (a.cin * 8 + 15) / 16;
    if (MT == 2 && J == 2)
      ptc_layer_tc_kernel<2, 2><<<a.b.total_blocks, 4 * PTC_SITES_PER_CTA, 0, st>>>(a, frag);
    else if (MT == 2 && J == 1)
      ptc_layer_tc_kernel<2, 1><<<a.b.total_blocks, 4 * PTC_SITES_PER_CTA, 0, st>>>(a, frag);
    else if (MT == 1 && J == 2)
      ptc_layer_tc_kernel<1, 2><<<a.b.total_blocks, 4 * PTC_SITES_PER_CTA, 0, st>>>(a, frag);
    else
      ptc_layer_tc_kernel<1, 1><<<a.b.total_blocks, 4 * PTC_SITES_PER_CTA, 0, st>>>(a, frag);
  } else {
    ptc_layer_kernel<<<a.b.total_blocks, 4 * PTC_SITES_PER_CTA, 0, st>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// weight gradient: block (slice chunk, ci*9 + s); every thread sums its sites
// of G_co(x) (T_s in_ci)(x)^+ into 16*COUT complex registers, the block reduces
template <int COUT>
__global__ void __launch_bounds__(128) ptc_grad_kernel(const __grid_constant__ PtcGradArgs a) {
  const Slice s = find_slice(a.b, blockIdx.x);
  const LatGeom& g = a.b.lat[s.l];
  const int cs = blockIdx.y;  // ci * 9 + shift
  const int ci = cs / PTC_NSHIFT, sh = cs % PTC_NSHIFT;
  const long stride = g.stride;
  const int p = a.parity;
  const void* g_here = a.gauge[s.l][p];
  const void* g_there = a.gauge[s.l][1 - p];
  const float4* f_here = a.in[s.l] + ptc_field_offset(s.rhs, ci, a.cin, p, stride);
  const float4* f_there = a.in[s.l] + ptc_field_offset(s.rhs, ci, a.cin, 1 - p, stride);

  float acc[COUT * 32];
#pragma unroll
  for (int k = 0; k < COUT * 32; k++) acc[k] = 0.f;
  for (long i = (long)s.chunk * blockDim.x + threadIdx.x; i < g.vh; i += (long)g.nchunk * blockDim.x) {
    const Nbr n = neighbours(g, p, i);
    cpx<float> t[12];
    transport(t, sh, f_here, f_there, g_here, g_there, stride, i, n);
#pragma unroll
    for (int co = 0; co < COUT; co++) {
      cpx<float> gv[12];
      SpinorIO<F32>::load(gv, a.g[s.l] + ptc_field_offset(s.rhs, co, COUT, p, stride), nullptr, stride, i);
#pragma unroll
      for (int al = 0; al < 4; al++)
#pragma unroll
        for (int be = 0; be < 4; be++) {
          cpx<float> v = {acc[co * 32 + (al * 4 + be) * 2], acc[co * 32 + (al * 4 + be) * 2 + 1]};
#pragma unroll
          for (int col = 0; col < 3; col++) cfma_conj(v, t[3 * be + col], gv[3 * al + col]);
          acc[co * 32 + (al * 4 + be) * 2] = v.re;
          acc[co * 32 + (al * 4 + be) * 2 + 1] = v.im;
        }
    }
  }
  // block reduction: warp shuffles, then one partial per block in FP64
  __shared__ double sh_acc[4][PTC_MAXC * 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < COUT * 32; k++) {
    float v = acc[k];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh_acc[warp][k] = v;
  }
  __syncthreads();
  double2* dst = a.partials + (((size_t)s.slot * (a.cin * PTC_NSHIFT) + cs) * a.maxch + s.chunk) * (COUT * 16);
  for (int k = threadIdx.x; k < COUT * 16; k += blockDim.x) {
    double re = 0, im = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      re += sh_acc[w][2 * k];
      im += sh_acc[w][2 * k + 1];
    }
    dst[k] = make_double2(re, im);
  }
}

cudaError_t ptc_grad(const PtcGradArgs& a, int block, cudaStream_t st) {
  dim3 grid(a.b.total_blocks, a.cin * PTC_NSHIFT);
  if (a.cout == 1)
    ptc_grad_kernel<1><<<grid, block, 0, st>>>(a);
  else if (a.cout == 4)
    ptc_grad_kernel<4><<<grid, block, 0, st>>>(a);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace wcl
