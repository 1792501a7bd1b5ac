// PTC network layer and weight-gradient kernels (see ptc.cuh).
#include "blackwell.cuh"
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
// Fifth-generation tensor-core layer (tcgen05, BF16 weights).  One CTA per tile of 128
// sites of one (lattice, rhs) slice and output parity; the sites are the M = 128 rows
// of the MMA.  For every shift s and colour c the mixing is the real GEMM
//   D_c[site][(co, alpha, re/im)] += sum_k X_{s,c}[site][k] B_s[(co, alpha, re/im)][k],
//   k = (ci, beta, re/im),
// with B_s the weights W[co][ci][s] in real form [[Re, -Im], [Im, Re]] (exact in BF16;
// N = 8 cout and K = 8 cin, each padded to 16) and X_{s,c} the transported inputs of
// colour c, split into NPART BF16 terms (hi + mid + lo carry 24 significant bits), each
// its own K block of the same B.  The SIMT threads compute the transports (gathers and
// link multiplies, as in the layers above) and write X in the no-swizzle K-major
// core-matrix layout of blackwell.cuh, where the eight values (beta, re/im) of one
// (site, ci, colour) are exactly one 16-byte core-matrix row.  One thread issues the
// 3 x NPART x K/16 MMAs of a shift (descriptors into shared memory, accumulators in
// tensor memory: colour c in columns [c N, (c + 1) N)) and commits them to an mbarrier;
// the X buffer is rewritten for the next shift once that mbarrier's phase completes,
// with the next shift's gathers already issued.  After the ninth shift every warp
// reads its lane quarter of the accumulators (tcgen05.ld) and stores whole spinors of
// one output channel.  Every mbarrier wait is bounded: on expiry the CTA stops issuing,
// waits (bounded) for its MMAs in flight, frees its tensor memory, sets bit 0x200 of
// the error word and leaves its outputs unwritten.
constexpr int UPTC_SITES = 128;
constexpr int UPTC_THREADS = 256;
constexpr unsigned UPTC_TMEM_COLS = 128;  // 3 colours x N <= 96 columns
constexpr long UPTC_WAIT_LIMIT = 1L << 22;

__host__ __device__ inline int uptc_n(int cout) { return cout * 8 < 16 ? 16 : cout * 8; }
__host__ __device__ inline int uptc_k(int cin) { return cin * 8 < 16 ? 16 : cin * 8; }

// B operands of the nine shifts, [shift][N / 8][K / 8][8][8] BF16
__global__ void ptc_pack_umma_kernel(const __nv_bfloat162* __restrict__ wb, int cin, int cout,
                                     __nv_bfloat16* __restrict__ out) {
  const int nn = uptc_n(cout), kk = uptc_k(cin), per = nn * kk;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= PTC_NSHIFT * per) return;
  const int sh = e / per, r = e - sh * per;
  const int n = r / kk, k = r - n * kk;
  const int co = n >> 3, al = (n >> 1) & 3, ro = n & 1;
  const int ci = k >> 3, be = (k >> 1) & 3, ri = k & 1;
  float v = 0.f;
  if (co < cout && ci < cin) {
    const float2 w = __bfloat1622float2(wb[((co * cin + ci) * PTC_NSHIFT + sh) * 16 + al * 4 + be]);
    v = ro == 0 ? (ri == 0 ? w.x : -w.y) : (ri == 0 ? w.y : w.x);
  }
  out[sh * per + ((n >> 3) * (kk >> 3) + (k >> 3)) * 64 + (n & 7) * 8 + (k & 7)] = __float2bfloat16_rn(v);
}

// eight floats -> NPART rows of eight BF16 whose sum carries 8 NPART significant bits
template <int NPART>
__device__ __forceinline__ void split_row(const float v[8], uint4 out[NPART]) {
  float rest[8];
#pragma unroll
  for (int k = 0; k < 8; k++) rest[k] = v[k];
#pragma unroll
  for (int part = 0; part < NPART; part++) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(rest[2 * k], rest[2 * k + 1]);
      const float2 f = __bfloat1622float2(h);
      rest[2 * k] -= f.x;
      rest[2 * k + 1] -= f.y;
      w[k] = bf16x2_bits(h);
    }
    out[part] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int NPART>
__global__ void __launch_bounds__(UPTC_THREADS, NPART == 3 ? 2 : NPART == 2 ? 3 : 4)
    ptc_layer_umma_kernel(const __grid_constant__ PtcLayerArgs a, const uint4* __restrict__ bpack, int* err) {
  extern __shared__ __align__(128) unsigned char uptc_smem[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  const int nn = uptc_n(a.cout), kk = uptc_k(a.cin);
  const int xbytes = UPTC_SITES * kk * 2;  // one (part, colour) X operand
  const int bshift = nn * kk * 2;          // one shift's B operand
  unsigned char* X = uptc_smem;
  unsigned char* Bs = uptc_smem + NPART * 3 * xbytes;
  // K columns of absent input channels stay zero; B is copied once for all shifts
  for (int k = threadIdx.x; k < NPART * 3 * xbytes / 16; k += blockDim.x)
    reinterpret_cast<uint4*>(X)[k] = make_uint4(0u, 0u, 0u, 0u);
  for (int k = threadIdx.x; k < PTC_NSHIFT * bshift / 16; k += blockDim.x) reinterpret_cast<uint4*>(Bs)[k] = bpack[k];
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  if (threadIdx.x < 32) tmem_alloc(&tslot, UPTC_TMEM_COLS);
  tc_fence_before_sync();
  __syncthreads();
  tc_fence_after_sync();
  const uint32_t tbase = tslot;

  const Slice s = find_slice(a.b, blockIdx.x);
  const LatGeom& g = a.b.lat[s.l];
  const int row = threadIdx.x & (UPTC_SITES - 1), half = threadIdx.x >> 7;  // site row; channels half, half + 2
  const long i = (long)s.chunk * UPTC_SITES + row;
  const bool site_ok = i < g.vh;
  const long ii = site_ok ? i : 0;
  const long stride = g.stride;
  const int p = a.parity;
  const Nbr n = neighbours(g, p, ii);
  const void* g_here = a.gauge[s.l][p];
  const void* g_there = a.gauge[s.l][1 - p];
  // byte offset of this site's row in K group 0 of an X operand
  const int xrow = ((row >> 3) * (kk >> 3)) * 128 + (row & 7) * 16;
  const uint32_t idesc = idesc_bf16_f32(UPTC_SITES, nn);
  const unsigned x0 = smem_u32(X), b0 = smem_u32(Bs), sbo = (unsigned)(kk >> 3) * 128u;

  auto put = [&](const cpx<float> t[12], int ci) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      float v[8];
#pragma unroll
      for (int be = 0; be < 4; be++) {
        v[2 * be] = t[3 * be + c].re;
        v[2 * be + 1] = t[3 * be + c].im;
      }
      uint4 parts[NPART];
      split_row<NPART>(v, parts);
#pragma unroll
      for (int part = 0; part < NPART; part++)
        *reinterpret_cast<uint4*>(X + (part * 3 + c) * xbytes + xrow + ci * 128) = parts[part];
    }
  };
  auto fetch = [&](cpx<float> t[12], int sh, int ci) {
    if (site_ok) {
      const float4* fh = a.in[s.l] + ptc_field_offset(s.rhs, ci, a.cin, p, stride);
      const float4* ft = a.in[s.l] + ptc_field_offset(s.rhs, ci, a.cin, 1 - p, stride);
      transport(t, sh, fh, ft, g_here, g_there, stride, ii, n);
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) t[k] = {0.f, 0.f};
    }
  };

  int issued = 0;  // shifts whose MMAs were committed
  bool ok = true;
#pragma unroll 1
  for (int sh = 0; sh < PTC_NSHIFT; sh++) {
    int timeout = 0;
    cpx<float> t[12];
    if (half < a.cin) fetch(t, sh, half);
    // the X buffer is free once the previous shift's MMAs have completed
    if (sh > 0 && !mbar_wait_bounded(&bar, (unsigned)(sh - 1) & 1u, UPTC_WAIT_LIMIT)) timeout = 1;
    if (!timeout) {
      if (half < a.cin) put(t, half);
      if (half + 2 < a.cin) {
        fetch(t, sh, half + 2);
        put(t, half + 2);
      }
    }
    fence_proxy_async();  // X written by ordinary stores, read by the tensor core
    tc_fence_before_sync();
    if (__syncthreads_or(timeout)) {
      ok = false;
      break;
    }
    tc_fence_after_sync();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int c = 0; c < 3; c++)
#pragma unroll
        for (int part = 0; part < NPART; part++)
          for (int j = 0; j < (kk >> 4); j++) {
            const uint64_t ad = make_smem_desc(x0 + (unsigned)((part * 3 + c) * xbytes + j * 256), 128u, sbo);
            const uint64_t bd = make_smem_desc(b0 + (unsigned)(sh * bshift + j * 256), 128u, sbo);
            umma_bf16(tbase + (uint32_t)(c * nn), ad, bd, idesc, (sh | part | j) != 0);
          }
      umma_commit(&bar);
    }
    issued++;
  }
  // the last committed phase: every MMA of the CTA has completed
  if (issued > 0 && !mbar_wait_bounded(&bar, (unsigned)(issued - 1) & 1u, UPTC_WAIT_LIMIT)) ok = false;
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after_sync();
  if (ok) {
    const uint32_t lane_base = (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16;
#pragma unroll 1
    for (int co = half; co < a.cout; co += 2) {
      float v[3][8];
#pragma unroll
      for (int c = 0; c < 3; c++) tmem_ld8(tbase + lane_base + (uint32_t)(c * nn + co * 8), v[c]);
      tmem_ld_wait();
      cpx<float> o12[12];
#pragma unroll
      for (int al = 0; al < 4; al++)
#pragma unroll
        for (int c = 0; c < 3; c++) o12[3 * al + c] = {v[c][2 * al], v[c][2 * al + 1]};
      if (site_ok) {
        float4* o = a.out[s.l] + ptc_field_offset(s.rhs, co, a.cout, p, stride);
        if (a.accumulate) {
          cpx<float> prev[12];
          SpinorIO<F32>::load<false>(prev, o, nullptr, stride, i);
#pragma unroll
          for (int k = 0; k < 12; k++) o12[k] = o12[k] + prev[k];
        }
        SpinorIO<F32>::store(o12, o, nullptr, stride, i);
      }
    }
  } else if (threadIdx.x == 0) {
    atomicOr(err, 0x200);
  }
  tc_fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after_sync();
    tmem_dealloc(tbase, UPTC_TMEM_COLS);
  }
}

int ptc_umma_sites_per_cta() { return UPTC_SITES; }
size_t ptc_umma_pack_bytes(int cin, int cout) { return (size_t)PTC_NSHIFT * uptc_n(cout) * uptc_k(cin) * 2; }

cudaError_t ptc_pack_umma(const __nv_bfloat162* wb, int cin, int cout, uint4* out, cudaStream_t st) {
  const int n = PTC_NSHIFT * uptc_n(cout) * uptc_k(cin);
  ptc_pack_umma_kernel<<<(n + 255) / 256, 256, 0, st>>>(wb, cin, cout, reinterpret_cast<__nv_bfloat16*>(out));
  return cudaGetLastError();
}

template <int NPART>
static cudaError_t launch_umma(const PtcLayerArgs& a, const uint4* bpack, int* err, cudaStream_t st) {
  const size_t smem = (size_t)NPART * 3 * UPTC_SITES * uptc_k(a.cin) * 2 + ptc_umma_pack_bytes(a.cin, a.cout);
  cudaError_t e = cudaFuncSetAttribute(ptc_layer_umma_kernel<NPART>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  ptc_layer_umma_kernel<NPART><<<a.b.total_blocks, UPTC_THREADS, smem, st>>>(a, bpack, err);
  return cudaGetLastError();
}

cudaError_t ptc_layer_umma(const PtcLayerArgs& a, const uint4* bpack, int nparts, int* err, cudaStream_t st) {
  if (a.cout < 1 || a.cout > PTC_MAXC || a.cin < 1 || a.cin > PTC_MAXC || !bpack || !err) return cudaErrorInvalidValue;
  if (nparts == 1) return launch_umma<1>(a, bpack, err, st);
  if (nparts == 2) return launch_umma<2>(a, bpack, err, st);
  if (nparts == 3) return launch_umma<3>(a, bpack, err, st);
  return cudaErrorInvalidValue;
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
