// Two-level adaptive aggregation multigrid for the Wilson-clover operator M of Eq. 5
// on the whole lattice: the solver QUDA provides and the paper enables through its
// multigrid parameters (Sec. II.E; Sec. III.B passes one geometric block size per
// level).  The paper names the method without its steps; the steps here are the
// standard aggregation ones, the same as the FP64 oracle's:
//
//   null space   N_v start vectors relaxed towards M x = 0 by minimal-residual steps
//                (r = -M x; alpha = <M r, r>/|M r|^2; x += alpha r; r -= alpha M r),
//                each then normalised;
//   prolongator  per coarse site (one block of b_x b_y b_z b_t fine sites) and per
//                chirality (spins {0,1} / {2,3}, the gamma_5 eigenspaces of the
//                DeGrand-Rossi basis) the restrictions of the null vectors made
//                orthonormal (modified Gram-Schmidt, applied twice): P^+ P = 1 and P
//                commutes with gamma_5;
//   coarse op    A_c = P^+ M P as a nine-point stencil of (2 N_v) x (2 N_v) blocks,
//                X(c) c(c) + sum_mu Yf_mu(c) c(c + mu) + Yb_mu(c) c(c - mu), built
//                locally from the links, the clover term and P(x): X collects
//                P(x)^+ A(x) P(x) and the hops that stay inside the block, Yf / Yb
//                the hops across the block's upper / lower face in mu;
//   K-cycle      minimal-residual pre-smoothing from zero, coarse correction
//                P A_c^-1 P^+ (r - M e) with the coarse system solved by GCR to a
//                relative tolerance, minimal-residual post-smoothing;
//   outer solve  flexible GCR (modified Gram-Schmidt) preconditioned by one K-cycle,
//                in FP32, restarted from the IEEE FP64 true residual of the whole
//                system until ||b - M x|| / ||b|| reaches the tolerance.
//
// Everything runs in this file's kernels and the library's fused dslash kernels;
// scalar coefficients (dot products summed in a fixed order from per-block FP64
// partials) go through the host.  Layouts:
//   fine FP32 field   the library's F32 parity layout, even then odd parity in one
//                     buffer (6 float4 chunks x stride per parity);
//   P                 [parity][cb site][chirality][6][N_v] complex float, row d =
//                     3 * (spin - 2 chirality) + colour;
//   coarse vector     [Ct][Cz][Cy][Cx][chirality][N_v] complex float (lexicographic);
//   stencil           [9][coarse site][column b][row a] complex float, block 0 = X,
//                     1 + 2 mu = Yf_mu, 2 + 2 mu = Yb_mu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "context.cuh"

wcl_status wcl_enter(wcl_ctx* c);
wcl_status wcl_leave(wcl_ctx* c, wcl_status s);
bool wcl_resolve_field(const wcl_ctx* c, const void* p, const void** out, const char* what);

namespace wcl {

constexpr int MG_MAX_NV = 32;
constexpr int MG_MAX_N = 2 * MG_MAX_NV;

// geometry of one fine lattice and its blocking
struct MgGeom {
  int dims[4];   // Lx, Ly, Lz, Lt
  int lxh;
  long stride;   // padded sites per parity
  int block[4];  // bx, by, bz, bt
  int cdims[4];  // Cx, Cy, Cz, Ct
  int bsites;    // sites per block
  long nc;       // coarse sites
  int nv, n;     // null vectors, 2 nv
};

__host__ __device__ __forceinline__ long mg_cb(const MgGeom& g, int x, int y, int z, int t) {
  return (((long)t * g.dims[2] + z) * g.dims[1] + y) * g.lxh + x / 2;
}
// fine coordinates of block-local site s (x fastest) of coarse site c (x fastest)
__host__ __device__ __forceinline__ void mg_site(const MgGeom& g, long c, int s, int xyzt[4]) {
  long q = c;
  int cc[4];
  for (int d = 0; d < 4; d++) {
    cc[d] = (int)(q % g.cdims[d]);
    q /= g.cdims[d];
  }
  int r = s;
  for (int d = 0; d < 4; d++) {
    const int sd = r % g.block[d];
    r /= g.block[d];
    xyzt[d] = cc[d] * g.block[d] + sd;
  }
}
__host__ __device__ __forceinline__ long mg_coarse_of(const MgGeom& g, const int xyzt[4]) {
  long c = 0;
  for (int d = 3; d >= 0; d--) c = c * g.cdims[d] + xyzt[d] / g.block[d];
  return c;
}
// complex float value m (0..11, 3 spin + colour) of site (p, i) of a fine FP32 field
__device__ __forceinline__ float2 fine_get(const float4* v, long stride, int p, long i, int m) {
  const float4 q = v[((long)p * 6 + m / 2) * stride + i];
  return (m & 1) ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
}

// ---------------------------------------------------------------------------
// BLAS on complex float arrays (fine fields are float4 = two complex numbers)
__global__ void mg_cdot_kernel(const float2* __restrict__ a, const float2* __restrict__ b, long n,
                               double* __restrict__ part) {
  double re = 0, im = 0;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const float2 x = a[k], y = b[k];
    re += (double)x.x * y.x + (double)x.y * y.y;  // conj(a) b
    im += (double)x.x * y.y - (double)x.y * y.x;
  }
  __shared__ double sh[2][32];
  re = warp_sum(re);
  im = warp_sum(im);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = re;
    sh[1][w] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0, s = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
      r += sh[0][k];
      s += sh[1][k];
    }
    part[2 * blockIdx.x] = r;
    part[2 * blockIdx.x + 1] = s;
  }
}
// y = a x + y (complex a), or with scale_y: y = a x + b y
__global__ void mg_caxpby_kernel(float2* __restrict__ y, const float2* __restrict__ x, float2 a, float2 b, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const float2 u = x[k], v = y[k];
    y[k] = make_float2(a.x * u.x - a.y * u.y + b.x * v.x - b.y * v.y, a.x * u.y + a.y * u.x + b.x * v.y + b.y * v.x);
  }
}

// ---------------------------------------------------------------------------
// prolongator: copy null vector k into column k, then orthonormalise per block-chirality
__global__ void mg_fill_kernel(const float4* __restrict__ v, int k, MgGeom g, float2* __restrict__ P) {
  const long nsite = 2 * g.stride;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < nsite * 12; q += (long)gridDim.x * blockDim.x) {
    const long site = q / 12;
    const int m = (int)(q % 12);
    const int p = (int)(site / g.stride);
    const long i = site % g.stride;
    P[(site * 12 + m) * g.nv + k] = fine_get(v, g.stride, p, i, m);
  }
}

__device__ __forceinline__ long mg_row_addr(const MgGeom& g, long c, int chi, int row) {
  int x[4];
  mg_site(g, c, row / 6, x);
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long i = mg_cb(g, x[0], x[1], x[2], x[3]);
  return (((long)p * g.stride + i) * 12 + chi * 6 + row % 6) * g.nv;
}

__device__ __forceinline__ double2 block_sum2(double2 v, double2* sh) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double2 t = make_double2(0, 0);
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
    t.x += sh[k].x;
    t.y += sh[k].y;
  }
  return t;
}

// one CTA per (coarse site, chirality): modified Gram-Schmidt over the nv columns,
// twice (the second pass restores orthogonality lost to rounding); a column whose
// norm vanishes is left zero and reported in flags
__global__ void __launch_bounds__(256) mg_orthonormalize_kernel(float2* __restrict__ P, MgGeom g,
                                                               int* __restrict__ flags) {
  __shared__ double2 sh[32];
  const long c = blockIdx.x / 2;
  const int chi = blockIdx.x % 2;
  const int rows = g.bsites * 6;
  for (int j = 0; j < g.nv; j++) {
    for (int pass = 0; pass < 2; pass++) {
      for (int k = 0; k < j; k++) {
        double2 d = make_double2(0, 0);
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
          const long a = mg_row_addr(g, c, chi, r);
          const float2 u = P[a + k], v = P[a + j];
          d.x += (double)u.x * v.x + (double)u.y * v.y;
          d.y += (double)u.x * v.y - (double)u.y * v.x;
        }
        d = block_sum2(d, sh);
        for (int r = threadIdx.x; r < rows; r += blockDim.x) {
          const long a = mg_row_addr(g, c, chi, r);
          const float2 u = P[a + k], v = P[a + j];
          P[a + j] = make_float2((float)(v.x - (d.x * u.x - d.y * u.y)), (float)(v.y - (d.x * u.y + d.y * u.x)));
        }
        __syncthreads();
      }
    }
    double2 nn = make_double2(0, 0);
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      const float2 v = P[mg_row_addr(g, c, chi, r) + j];
      nn.x += (double)v.x * v.x + (double)v.y * v.y;
    }
    nn = block_sum2(nn, sh);
    const double inv = nn.x > 0 ? 1.0 / sqrt(nn.x) : 0.0;
    if (!(nn.x > 0) && threadIdx.x == 0) atomicOr(flags, 8);
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      const long a = mg_row_addr(g, c, chi, r);
      const float2 v = P[a + j];
      P[a + j] = make_float2((float)(v.x * inv), (float)(v.y * inv));
    }
    __syncthreads();
  }
}

// c = P^+ v: one CTA per (coarse site, right-hand side blockIdx.y); the block's fine
// values are staged in shared memory.  pstride: float4 elements between the two parities
// of one right-hand side (6 stride for one whole-lattice field, nrhs 6 stride for the
// batched layout); rfine / rcoarse: offsets between right-hand sides.
__global__ void __launch_bounds__(128) mg_restrict_kernel(const float4* __restrict__ v, const float2* __restrict__ P,
                                                         MgGeom g, float2* __restrict__ out, long pstride,
                                                         long rfine, long rcoarse) {
  extern __shared__ float2 vs[];  // [bsites][12]
  const long c = blockIdx.x;
  v += blockIdx.y * rfine;
  out += blockIdx.y * rcoarse;
  for (int q = threadIdx.x; q < g.bsites * 12; q += blockDim.x) {
    int x[4];
    mg_site(g, c, q / 12, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const int m = q % 12;
    const float4 f = v[p * pstride + (long)(m / 2) * g.stride + mg_cb(g, x[0], x[1], x[2], x[3])];
    vs[q] = (m & 1) ? make_float2(f.z, f.w) : make_float2(f.x, f.y);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < g.n; j += blockDim.x) {
    const int chi = j / g.nv, k = j % g.nv;
    double re = 0, im = 0;
    for (int s = 0; s < g.bsites; s++) {
      int x[4];
      mg_site(g, c, s, x);
      const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
      const long base = ((long)p * g.stride + mg_cb(g, x[0], x[1], x[2], x[3])) * 12;
#pragma unroll
      for (int d = 0; d < 6; d++) {
        const float2 u = P[(base + chi * 6 + d) * g.nv + k], w = vs[s * 12 + chi * 6 + d];
        re += (double)u.x * w.x + (double)u.y * w.y;
        im += (double)u.x * w.y - (double)u.y * w.x;
      }
    }
    out[c * g.n + j] = make_float2((float)re, (float)im);
  }
}

// v = P c (accumulate: v += P c): one thread per fine site, right-hand side blockIdx.y
// (pstride, rfine, rcoarse as for mg_restrict_kernel)
__global__ void mg_prolong_kernel(const float2* __restrict__ cvec, const float2* __restrict__ P, MgGeom g,
                                  float4* __restrict__ v, int accumulate, long pstride, long rfine, long rcoarse) {
  const long vh = g.stride;  // padded sites per parity; padding rows of P are zero
  cvec += blockIdx.y * rcoarse;
  v += blockIdx.y * rfine;
  for (long site = blockIdx.x * (long)blockDim.x + threadIdx.x; site < 2 * vh;
       site += (long)gridDim.x * blockDim.x) {
    const int p = (int)(site / vh);
    const long i = site % vh;
    // coordinates of (p, i)
    const int xh = (int)(i % g.lxh);
    long rem = i / g.lxh;
    const int y = (int)(rem % g.dims[1]);
    rem /= g.dims[1];
    const int z = (int)(rem % g.dims[2]);
    const int t = (int)(rem / g.dims[2]);
    if (t >= g.dims[3]) continue;  // padding
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const int xyzt[4] = {x, y, z, t};
    const long c = mg_coarse_of(g, xyzt);
    float2 o[12];
#pragma unroll
    for (int m = 0; m < 12; m++) {
      const int chi = m / 6;
      double re = 0, im = 0;
      for (int k = 0; k < g.nv; k++) {
        const float2 u = P[(site * 12 + m) * g.nv + k], w = cvec[c * g.n + chi * g.nv + k];
        re += (double)u.x * w.x - (double)u.y * w.y;
        im += (double)u.x * w.y + (double)u.y * w.x;
      }
      o[m] = make_float2((float)re, (float)im);
    }
#pragma unroll
    for (int q = 0; q < 6; q++) {
      float4* dst = v + p * pstride + (long)q * vh + i;
      float4 val = make_float4(o[2 * q].x, o[2 * q].y, o[2 * q + 1].x, o[2 * q + 1].y);
      if (accumulate) {
        const float4 old = *dst;
        val = make_float4(old.x + val.x, old.y + val.y, old.z + val.z, old.w + val.w);
      }
      *dst = val;
    }
  }
}

// ---------------------------------------------------------------------------
// coarse operator: one CTA per (coarse site, block q); q = 0 X, 1 + 2 mu Yf_mu, 2 + 2 mu Yb_mu
struct MgBuildArgs {
  MgGeom g;
  const void* gauge[2];  // FP32 links per parity
  const void* clov[2];   // FP32 clover A per parity
  double kappa;          // hopping parameter of the library's operator (kappa nu / xi_0 anisotropic)
  float tw_f, tbw_f;     // t-hop weight inside the lattice / across the time boundary
  const float2* P;
  float2* Y;             // [9][nc][n (column)][n (row)]
};

// T[:, j] = -kappa w eta (1 -/+ gamma_mu) U P(nbr)[:, j] for hop (mu, back) from site (p, i)
template <int MU, bool BACK>
__device__ void mg_hop_columns(const MgBuildArgs& a, int p, long i, const int x[4], float2* T, int n) {
  const MgGeom& g = a.g;
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[MU] = BACK ? (x[MU] == 0 ? g.dims[MU] - 1 : x[MU] - 1) : (x[MU] + 1 == g.dims[MU] ? 0 : x[MU] + 1);
  const int pn = 1 - p;
  const long in_ = mg_cb(g, y[0], y[1], y[2], y[3]);
  float w = 1.f;
  if (MU == 3) {
    const bool edge = BACK ? (x[3] == 0) : (x[3] + 1 == g.dims[3]);
    w = edge ? a.tbw_f : a.tw_f;
  }
  const float coef = (float)(-a.kappa) * w;
  cpx<float> u[3][3];
  if (BACK)
    LinkIO<F32>::load(u, a.gauge[pn], g.stride, in_, MU);  // U_mu(x - mu), used as U^+
  else
    LinkIO<F32>::load(u, a.gauge[p], g.stride, i, MU);
  constexpr int S = BACK ? +1 : -1;  // projector 1 + S gamma_mu
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    cpx<float> psi[12], h[6], uh[6], out[12];
    const long pb = ((long)pn * g.stride + in_) * 12;
#pragma unroll
    for (int m = 0; m < 12; m++) {
      const float2 v = a.P[(pb + m) * g.nv + (j % g.nv)];
      // column j of P(nbr) lives in chirality j / nv only
      const bool on = (m / 6) == (j / g.nv);
      psi[m] = on ? cpx<float>{v.x, v.y} : cpx<float>{0.f, 0.f};
    }
#pragma unroll
    for (int m = 0; m < 12; m++) out[m] = {0.f, 0.f};
    project<MU, S>(psi, h);
    link_mul<BACK>(u, h, uh, coef);
    reconstruct_acc<MU, S>(out, uh);
#pragma unroll
    for (int m = 0; m < 12; m++) T[m * n + j] = make_float2(out[m].re, out[m].im);
  }
}

__device__ void mg_hop_dispatch(const MgBuildArgs& a, int mu, bool back, int p, long i, const int x[4], float2* T,
                                int n) {
  switch (mu * 2 + (back ? 1 : 0)) {
    case 0: mg_hop_columns<0, false>(a, p, i, x, T, n); break;
    case 1: mg_hop_columns<0, true>(a, p, i, x, T, n); break;
    case 2: mg_hop_columns<1, false>(a, p, i, x, T, n); break;
    case 3: mg_hop_columns<1, true>(a, p, i, x, T, n); break;
    case 4: mg_hop_columns<2, false>(a, p, i, x, T, n); break;
    case 5: mg_hop_columns<2, true>(a, p, i, x, T, n); break;
    case 6: mg_hop_columns<3, false>(a, p, i, x, T, n); break;
    default: mg_hop_columns<3, true>(a, p, i, x, T, n); break;
  }
}

constexpr int MG_BUILD_THREADS = 256;
constexpr int MG_BUILD_PER = MG_MAX_N * MG_MAX_N / MG_BUILD_THREADS;  // entries per thread (16)

__global__ void __launch_bounds__(MG_BUILD_THREADS) mg_build_kernel(const __grid_constant__ MgBuildArgs a) {
  const MgGeom& g = a.g;
  const int n = g.n;
  const long c = blockIdx.x / 9;
  const int q = blockIdx.x % 9;
  extern __shared__ float2 sm[];
  float2* Px = sm;           // [12][n]
  float2* T = sm + 12 * n;   // [12][n]
  float2 acc[MG_BUILD_PER];
#pragma unroll
  for (int e = 0; e < MG_BUILD_PER; e++) acc[e] = make_float2(0.f, 0.f);
  for (int s = 0; s < g.bsites; s++) {
    int x[4];
    mg_site(g, c, s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const long i = mg_cb(g, x[0], x[1], x[2], x[3]);
    // the terms of site x that land in block q
    int nterm = 0, terms[9];
    if (q == 0) {
      terms[nterm++] = -1;  // clover
      for (int mu = 0; mu < 4; mu++) {
        const int sd = x[mu] % g.block[mu];
        if (sd != g.block[mu] - 1) terms[nterm++] = 2 * mu;
        if (sd != 0) terms[nterm++] = 2 * mu + 1;
      }
    } else {
      const int mu = (q - 1) / 2;
      const bool back = ((q - 1) & 1) != 0;
      const int sd = x[mu] % g.block[mu];
      if (!back && sd == g.block[mu] - 1) terms[nterm++] = 2 * mu;
      if (back && sd == 0) terms[nterm++] = 2 * mu + 1;
    }
    if (nterm == 0) continue;
    __syncthreads();
    const long pb = ((long)p * g.stride + i) * 12;
    for (int e = threadIdx.x; e < 12 * n; e += blockDim.x) {
      const int m = e / n, j = e % n;
      const float2 v = a.P[(pb + m) * g.nv + (j % g.nv)];
      Px[e] = ((m / 6) == (j / g.nv)) ? v : make_float2(0.f, 0.f);
    }
    for (int t = 0; t < nterm; t++) {
      __syncthreads();
      if (terms[t] < 0) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          cpx<float> xin[12], yout[12];
#pragma unroll
          for (int m = 0; m < 12; m++) {
            const float2 v = Px[m * n + j];
            xin[m] = {v.x, v.y};
          }
          CloverIO<F32>::apply(yout, xin, a.clov[p], nullptr, g.stride, i);
#pragma unroll
          for (int m = 0; m < 12; m++) T[m * n + j] = make_float2(yout[m].re, yout[m].im);
        }
      } else {
        mg_hop_dispatch(a, terms[t] / 2, terms[t] & 1, p, i, x, T, n);
      }
      __syncthreads();
      // acc(row a, col b) += sum_m conj(Px[m][a]) T[m][b]
#pragma unroll
      for (int e = 0; e < MG_BUILD_PER; e++) {
        const int idx = threadIdx.x + e * MG_BUILD_THREADS;
        if (idx < n * n) {
          const int ra = idx % n, cb = idx / n;
          float re = acc[e].x, im = acc[e].y;
#pragma unroll
          for (int m = 0; m < 12; m++) {
            const float2 u = Px[m * n + ra], w = T[m * n + cb];
            re = fmaf(u.x, w.x, fmaf(u.y, w.y, re));
            im = fmaf(u.x, w.y, fmaf(-u.y, w.x, im));
          }
          acc[e] = make_float2(re, im);
        }
      }
    }
  }
  float2* out = a.Y + ((long)q * g.nc + c) * n * n;
#pragma unroll
  for (int e = 0; e < MG_BUILD_PER; e++) {
    const int idx = threadIdx.x + e * MG_BUILD_THREADS;
    if (idx < n * n) out[idx] = acc[e];  // [column cb][row ra]
  }
}

// out = A_c in: one CTA per coarse site, thread = output row; the nine input vectors
// (the site and its eight neighbours) are staged in shared memory
__global__ void __launch_bounds__(MG_MAX_N) mg_coarse_apply_kernel(const float2* __restrict__ Y,
                                                                  const float2* __restrict__ in, MgGeom g,
                                                                  float2* __restrict__ out) {
  __shared__ float2 vin[9][MG_MAX_N];
  const long c = blockIdx.x;
  const int n = g.n;
  int cc[4];
  long q = c;
  for (int d = 0; d < 4; d++) {
    cc[d] = (int)(q % g.cdims[d]);
    q /= g.cdims[d];
  }
  for (int e = threadIdx.x; e < 9 * n; e += blockDim.x) {
    const int k = e / n, b = e % n;
    int dd[4] = {cc[0], cc[1], cc[2], cc[3]};
    if (k > 0) {
      const int mu = (k - 1) / 2;
      const bool back = ((k - 1) & 1) != 0;
      dd[mu] = back ? (dd[mu] == 0 ? g.cdims[mu] - 1 : dd[mu] - 1) : (dd[mu] + 1 == g.cdims[mu] ? 0 : dd[mu] + 1);
    }
    long cn = 0;
    for (int d = 3; d >= 0; d--) cn = cn * g.cdims[d] + dd[d];
    vin[k][b] = in[cn * n + b];
  }
  __syncthreads();
  const int ra = threadIdx.x;
  if (ra >= n) return;
  float re = 0.f, im = 0.f;
  for (int k = 0; k < 9; k++) {
    const float2* blk = Y + ((long)k * g.nc + c) * n * n;
    for (int b = 0; b < n; b++) {
      const float2 y = blk[b * n + ra], v = vin[k][b];
      re = fmaf(y.x, v.x, fmaf(-y.y, v.y, re));
      im = fmaf(y.x, v.y, fmaf(y.y, v.x, im));
    }
  }
  out[c * n + ra] = make_float2(re, im);
}

// ---------------------------------------------------------------------------
// Batched K-cycle: nrhs right-hand sides at once, every coefficient on the device.
// Batched fine fields: [parity][rhs][6][stride] float4 (the even half of all right-hand
// sides is the library's nrhs parity field); batched coarse vectors [rhs][nc][n].

// out_r = A_c in_r for MGB_RB right-hand sides per pass: the stencil block of a coarse
// site is read once per pass instead of once per right-hand side
constexpr int MGB_RB = 6;
__global__ void __launch_bounds__(MG_MAX_N) mgb_coarse_apply_kernel(const float2* __restrict__ Y,
                                                                   const float2* __restrict__ in, MgGeom g,
                                                                   float2* __restrict__ out, int nrhs) {
  __shared__ float2 vin[9][MGB_RB][MG_MAX_N];
  const long c = blockIdx.x;
  const int n = g.n;
  const long rs = g.nc * n;
  int cc[4];
  long q = c;
  for (int d = 0; d < 4; d++) {
    cc[d] = (int)(q % g.cdims[d]);
    q /= g.cdims[d];
  }
  long cn[9];
  for (int k = 0; k < 9; k++) {
    int dd[4] = {cc[0], cc[1], cc[2], cc[3]};
    if (k > 0) {
      const int mu = (k - 1) / 2;
      const bool back = ((k - 1) & 1) != 0;
      dd[mu] = back ? (dd[mu] == 0 ? g.cdims[mu] - 1 : dd[mu] - 1) : (dd[mu] + 1 == g.cdims[mu] ? 0 : dd[mu] + 1);
    }
    long v = 0;
    for (int d = 3; d >= 0; d--) v = v * g.cdims[d] + dd[d];
    cn[k] = v;
  }
  for (int r0 = 0; r0 < nrhs; r0 += MGB_RB) {
    const int nr = min(MGB_RB, nrhs - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < 9 * MGB_RB * n; e += blockDim.x) {
      const int k = e / (MGB_RB * n), rr = (e / n) % MGB_RB, b = e % n;
      vin[k][rr][b] = rr < nr ? in[(r0 + rr) * rs + cn[k] * n + b] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int ra = threadIdx.x;
    if (ra < n) {
      float re[MGB_RB], im[MGB_RB];
#pragma unroll
      for (int rr = 0; rr < MGB_RB; rr++) re[rr] = im[rr] = 0.f;
      for (int k = 0; k < 9; k++) {
        const float2* blk = Y + ((long)k * g.nc + c) * n * n;
        for (int b = 0; b < n; b++) {
          const float2 y = blk[b * n + ra];
#pragma unroll
          for (int rr = 0; rr < MGB_RB; rr++) {
            const float2 v = vin[k][rr][b];
            re[rr] = fmaf(y.x, v.x, fmaf(-y.y, v.y, re[rr]));
            im[rr] = fmaf(y.x, v.y, fmaf(y.y, v.x, im[rr]));
          }
        }
      }
      for (int rr = 0; rr < nr; rr++) out[(r0 + rr) * rs + c * n + ra] = make_float2(re[rr], im[rr]);
    }
  }
}

// c_r = P^+ v_r for the batched layout: one CTA per (coarse site, right-hand side) with
// the right-hand side fastest, so that the CTAs sharing a coarse site's rows of P run
// together and read them from L2; the block's site offsets are computed once; the
// MGB_RG groups of the CTA's threads each sum a quarter of the sites for every output
// (FP32 sums: a preconditioner step), then the groups' sums are added
constexpr int MGB_RG = 4;
__global__ void __launch_bounds__(MGB_RG * MG_MAX_N) mgb_restrict_kernel(const float4* __restrict__ v,
                                                                        const float2* __restrict__ P, MgGeom g,
                                                                        float2* __restrict__ out, int nrhs) {
  extern __shared__ float2 vs[];  // [bsites][12], then the sites' P row bases
  __shared__ float2 red[MGB_RG][MG_MAX_N];
  long* base = reinterpret_cast<long*>(vs + g.bsites * 12);
  const long c = blockIdx.x / nrhs;
  const int r = (int)(blockIdx.x % nrhs);
  const long half = 6 * g.stride;
  for (int s = threadIdx.x; s < g.bsites; s += blockDim.x) {
    int x[4];
    mg_site(g, c, s, x);
    const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    const long i = mg_cb(g, x[0], x[1], x[2], x[3]);
    base[s] = ((long)p * g.stride + i) * 12;
    const float4* src = v + ((long)p * nrhs + r) * half + i;
#pragma unroll
    for (int q = 0; q < 6; q++) {
      const float4 f = src[q * g.stride];
      vs[s * 12 + 2 * q] = make_float2(f.x, f.y);
      vs[s * 12 + 2 * q + 1] = make_float2(f.z, f.w);
    }
  }
  __syncthreads();
  const int j = threadIdx.x % MG_MAX_N, grp = threadIdx.x / MG_MAX_N;
  if (j < g.n) {
    const int chi = j / g.nv, k = j % g.nv;
    float re = 0.f, im = 0.f;
    for (int s = grp; s < g.bsites; s += MGB_RG) {
      const long b0 = base[s] + chi * 6;
#pragma unroll
      for (int d = 0; d < 6; d++) {
        const float2 u = P[(b0 + d) * g.nv + k], w = vs[s * 12 + chi * 6 + d];
        re = fmaf(u.x, w.x, fmaf(u.y, w.y, re));
        im = fmaf(u.x, w.y, fmaf(-u.y, w.x, im));
      }
    }
    red[grp][j] = make_float2(re, im);
  }
  __syncthreads();
  if (grp == 0 && j < g.n) {
    float2 t = red[0][j];
    for (int q = 1; q < MGB_RG; q++) t = make_float2(t.x + red[q][j].x, t.y + red[q][j].y);
    out[((long)r * g.nc + c) * g.n + j] = t;
  }
}

// v_r += P c_r for the batched layout: one thread per fine site applies each row of P,
// read once, to every right-hand side (FP32 sums of nv terms)
constexpr int MGB_MAXR = 12;
__global__ void __launch_bounds__(128) mgb_prolong_kernel(const float2* __restrict__ cvec, const float2* __restrict__ P,
                                                         MgGeom g, float4* __restrict__ v, int nrhs) {
  const long vh = g.stride;
  const long half = 6 * vh;
  const long rs = g.nc * g.n;
  for (long site = blockIdx.x * (long)blockDim.x + threadIdx.x; site < 2 * vh;
       site += (long)gridDim.x * blockDim.x) {
    const int p = (int)(site / vh);
    const long i = site % vh;
    const int xh = (int)(i % g.lxh);
    long rem = i / g.lxh;
    const int y = (int)(rem % g.dims[1]);
    rem /= g.dims[1];
    const int z = (int)(rem % g.dims[2]);
    const int t = (int)(rem / g.dims[2]);
    if (t >= g.dims[3]) continue;  // padding
    const int x = 2 * xh + ((p + y + z + t) & 1);
    const int xyzt[4] = {x, y, z, t};
    const long c = mg_coarse_of(g, xyzt);
    for (int q = 0; q < 6; q++) {
      const int chi = (2 * q) / 6;
      float2 a0[MGB_MAXR], a1[MGB_MAXR];
#pragma unroll
      for (int r = 0; r < MGB_MAXR; r++) a0[r] = a1[r] = make_float2(0.f, 0.f);
      const float2* p0 = P + (site * 12 + 2 * q) * g.nv;
      const float2* p1 = p0 + g.nv;
      const float2* cv = cvec + c * g.n + chi * g.nv;
      for (int k = 0; k < g.nv; k++) {
        const float2 u0 = p0[k], u1 = p1[k];
#pragma unroll
        for (int r = 0; r < MGB_MAXR; r++) {
          if (r >= nrhs) break;
          const float2 w = cv[r * rs + k];
          a0[r].x = fmaf(u0.x, w.x, fmaf(-u0.y, w.y, a0[r].x));
          a0[r].y = fmaf(u0.x, w.y, fmaf(u0.y, w.x, a0[r].y));
          a1[r].x = fmaf(u1.x, w.x, fmaf(-u1.y, w.y, a1[r].x));
          a1[r].y = fmaf(u1.x, w.y, fmaf(u1.y, w.x, a1[r].y));
        }
      }
#pragma unroll
      for (int r = 0; r < MGB_MAXR; r++) {
        if (r >= nrhs) break;
        float4* dst = v + ((long)p * nrhs + r) * half + (long)q * vh + i;
        const float4 old = *dst;
        *dst = make_float4(old.x + a0[r].x, old.y + a0[r].y, old.z + a1[r].x, old.w + a1[r].y);
      }
    }
  }
}

// The vector of right-hand side r is n complex numbers at r rstride and, with seg2 > 0,
// n more at seg2 + r rstride (the odd half of a batched fine field).
__device__ __forceinline__ long mgb_index(long k, long n, long off, long seg2) {
  return k < n ? off + k : seg2 + off + (k - n);
}

// per right-hand side r = blockIdx.y: partial sums of <a_r, b_r> and, with c, <a_r, c_r>
// (conj(a) b); part[((r * gridDim.x) + block) * 4 + {0..3}].  Each thread sums its
// elements in FP32 (GB300's FP64 rate made FP64 products the cost of this kernel), the
// threads' sums are added in FP64.
__global__ void __launch_bounds__(256) mgb_dot_kernel(const float2* __restrict__ a, const float2* __restrict__ b,
                                                      const float2* __restrict__ c, long n, long rstride, long seg2,
                                                      double* __restrict__ part) {
  const long off = blockIdx.y * rstride;
  const long ntot = seg2 > 0 ? 2 * n : n;
  float f[4] = {0.f, 0.f, 0.f, 0.f};
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < ntot; k += (long)gridDim.x * blockDim.x) {
    const long q = mgb_index(k, n, off, seg2);
    const float2 x = a[q], y = b[q];
    f[0] = fmaf(x.x, y.x, fmaf(x.y, y.y, f[0]));
    f[1] = fmaf(x.x, y.y, fmaf(-x.y, y.x, f[1]));
    if (c) {
      const float2 z = c[q];
      f[2] = fmaf(x.x, z.x, fmaf(x.y, z.y, f[2]));
      f[3] = fmaf(x.x, z.y, fmaf(-x.y, z.x, f[3]));
    }
  }
  double v[4] = {f[0], f[1], f[2], f[3]};
  __shared__ double sh[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const double t = warp_sum(v[j]);
    if (lane == 0) sh[j][w] = t;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[threadIdx.x][k];
    part[((long)blockIdx.y * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = t;
  }
}

// coefficients from the summed dots of right-hand side r = threadIdx.x (fixed order):
//   MGB_MR       alpha = <a,c> / <a,a>: ca = alpha, cb = -alpha    (minimal residual: a = M r, c = r)
//   MGB_PROJ     beta = <a,b>:          ca = -beta                  (Gram-Schmidt)
//   MGB_NORMINV  ca = 1 / sqrt(<a,a>)  (0 for a zero vector)
//   MGB_COEF     al = <a,b>:            ca = al, cb = -al
enum { MGB_MR = 0, MGB_PROJ = 1, MGB_NORMINV = 2, MGB_COEF = 3 };
__global__ void mgb_coef_kernel(const double* __restrict__ part, int nblk, int nrhs, int mode, float2* __restrict__ ca,
                                float2* __restrict__ cb) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  double s[4] = {0, 0, 0, 0};
  for (int k = 0; k < nblk; k++)
    for (int j = 0; j < 4; j++) s[j] += part[((long)r * nblk + k) * 4 + j];
  float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
  if (mode == MGB_MR) {
    if (s[0] > 0) {
      a = make_float2((float)(s[2] / s[0]), (float)(s[3] / s[0]));
      b = make_float2(-a.x, -a.y);
    }
  } else if (mode == MGB_PROJ) {
    a = make_float2((float)-s[0], (float)-s[1]);
  } else if (mode == MGB_NORMINV) {
    if (s[0] > 0) a = make_float2((float)(1.0 / sqrt(s[0])), 0.f);
  } else {
    a = make_float2((float)s[0], (float)s[1]);
    b = make_float2(-a.x, -a.y);
  }
  ca[r] = a;
  if (cb) cb[r] = b;
}

// y_r += coef[r] x_r (x given) or y_r = coef[r] y_r (x null), r = blockIdx.y
__global__ void mgb_axpy_kernel(float2* __restrict__ y, const float2* __restrict__ x, const float2* __restrict__ coef,
                                long n, long rstride, long seg2) {
  const long off = blockIdx.y * rstride;
  const long ntot = seg2 > 0 ? 2 * n : n;
  const float2 a = coef[blockIdx.y];
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < ntot; k += (long)gridDim.x * blockDim.x) {
    const long q = mgb_index(k, n, off, seg2);
    const float2 v = y[q];
    if (x) {
      const float2 u = x[q];
      y[q] = make_float2(v.x + a.x * u.x - a.y * u.y, v.y + a.x * u.y + a.y * u.x);
    } else {
      y[q] = make_float2(a.x * v.x - a.y * v.y, a.x * v.y + a.y * v.x);
    }
  }
}

// y = x - y elementwise (float2), the whole batch
__global__ void mgb_rsub_kernel(float2* __restrict__ y, const float2* __restrict__ x, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const float2 u = x[k], v = y[k];
    y[k] = make_float2(u.x - v.x, u.y - v.y);
  }
}

// ---------------------------------------------------------------------------
// FP64 full-field helpers for the defect correction (even then odd parity, F64 layout)
__global__ void mg_sub64_kernel(double2* __restrict__ r, const double2* __restrict__ b, const double2* __restrict__ y,
                                long n) {  // r = b - y
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    r[k] = make_double2(b[k].x - y[k].x, b[k].y - y[k].y);
}
__global__ void mg_norm64_kernel(const double2* __restrict__ a, long n, double* __restrict__ part) {
  double s = 0;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    s += a[k].x * a[k].x + a[k].y * a[k].y;
  __shared__ double sh[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
    part[blockIdx.x] = t;
  }
}
// FP64 (double2 per complex, 12 chunks per parity) -> FP32 (float4 per two complex)
__global__ void mg_to32_kernel(const double2* __restrict__ a, float4* __restrict__ o, long stride) {
  const long n = 2 * 6 * stride;  // float4 elements
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const long p = k / (6 * stride), rem = k % (6 * stride), ch = rem / stride, i = rem % stride;
    const double2 u = a[(p * 12 + 2 * ch) * stride + i], v = a[(p * 12 + 2 * ch + 1) * stride + i];
    o[k] = make_float4((float)u.x, (float)u.y, (float)v.x, (float)v.y);
  }
}
__global__ void mg_add32into64_kernel(double2* __restrict__ a, const float4* __restrict__ o, long stride) {
  const long n = 2 * 6 * stride;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const long p = k / (6 * stride), rem = k % (6 * stride), ch = rem / stride, i = rem % stride;
    const float4 f = o[k];
    double2& u = a[(p * 12 + 2 * ch) * stride + i];
    double2& v = a[(p * 12 + 2 * ch + 1) * stride + i];
    u = make_double2(u.x + f.x, u.y + f.y);
    v = make_double2(v.x + f.z, v.y + f.w);
  }
}

// ---------------------------------------------------------------------------
// host side

struct MgState {
  MgGeom g{};
  wcl_mg_params prm{};
  float2* P = nullptr;
  float2* Y = nullptr;
  float2* cw = nullptr;     // coarse workspace: x, r, 2 nkrylov (z, w)
  float4* fw = nullptr;     // fine FP32 workspace, MG_FINE fields
  double* part = nullptr;   // reduction partials (device)
  std::vector<double> hpart;
  bool ready = false;
};
constexpr int MG_FINE = 8;   // e, rr, ar, r1, t (cycle) + solve x, r, z (FGCR uses its own)
constexpr int MG_PART = 1024;

static int grid_of(long n) {
  long g = (n + 255) / 256;
  return (int)std::max(1L, std::min(g, 152L * 8));
}

static MgState* mg_of(wcl_ctx* c) { return static_cast<MgState*>(c->mg); }

void mg_free(wcl_ctx* c) {
  MgState* m = mg_of(c);
  if (!m) return;
  cudaFree(m->P);
  cudaFree(m->Y);
  cudaFree(m->cw);
  cudaFree(m->fw);
  cudaFree(m->part);
  delete m;
  c->mg = nullptr;
}

namespace {

struct Ctx {
  wcl_ctx* c;
  MgState* m;
  long nfine() const { return 2 * 12 * m->g.stride; }   // complex numbers in a fine FP32 field
  long ncoarse() const { return m->g.nc * m->g.n; }      // complex numbers in a coarse vector
  float4* fine(int k) const { return m->fw + (size_t)k * 2 * 6 * m->g.stride; }
  float2* coarse(int k) const { return m->cw + (size_t)k * m->g.nc * m->g.n; }

  wcl_status dot(const float2* a, const float2* b, long n, double2* out) {
    const int gb = std::min(MG_PART, grid_of(n));
    mg_cdot_kernel<<<gb, 256, 0, c->stream>>>(a, b, n, m->part);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    WCL_CUDA(cudaMemcpyAsync(m->hpart.data(), m->part, sizeof(double) * 2 * gb, cudaMemcpyDeviceToHost, c->stream));
    WCL_CUDA(cudaStreamSynchronize(c->stream));
    double re = 0, im = 0;
    for (int k = 0; k < gb; k++) {
      re += m->hpart[2 * k];
      im += m->hpart[2 * k + 1];
    }
    *out = make_double2(re, im);
    return WCL_OK;
  }
  wcl_status axpby(float2* y, const float2* x, double2 a, double2 b, long n) {
    mg_caxpby_kernel<<<grid_of(n), 256, 0, c->stream>>>(y, x, make_float2((float)a.x, (float)a.y),
                                                         make_float2((float)b.x, (float)b.y), n);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    return WCL_OK;
  }
  wcl_status copy(float2* y, const float2* x, long n) {
    WCL_CUDA(cudaMemcpyAsync(y, x, sizeof(float2) * n, cudaMemcpyDeviceToDevice, c->stream));
    return WCL_OK;
  }
  // fine FP32 M on the whole lattice: out_e = A x_e - kappa D x_o, out_o = A x_o - kappa D x_e
  wcl_status apply_M(float4* out, const float4* in) {
    std::vector<wcl_ctx*> v{c};
    const long half = 6 * m->g.stride;
    FieldRef ie{}, io{}, oe{}, oo{};
    ie.ptr[0] = const_cast<float4*>(in);
    io.ptr[0] = const_cast<float4*>(in) + half;
    oe.ptr[0] = out;
    oo.ptr[0] = out + half;
    WCL_CHECK(dslash(v, F32, 1, oe, io, &ie, 0, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, nullptr));
    WCL_CHECK(dslash(v, F32, 1, oo, ie, &io, 1, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, nullptr));
    return WCL_OK;
  }
  wcl_status restrict_(float2* out, const float4* in) {
    const size_t sm = sizeof(float2) * m->g.bsites * 12;
    mg_restrict_kernel<<<(unsigned)m->g.nc, 128, sm, c->stream>>>(in, m->P, m->g, out, 6 * m->g.stride, 0, 0);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    return WCL_OK;
  }
  wcl_status prolong(float4* out, const float2* in, bool accumulate) {
    mg_prolong_kernel<<<grid_of(2 * m->g.stride), 256, 0, c->stream>>>(in, m->P, m->g, out, accumulate ? 1 : 0,
                                                                      6 * m->g.stride, 0, 0);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    return WCL_OK;
  }
  wcl_status coarse_apply(float2* out, const float2* in) {
    mg_coarse_apply_kernel<<<(unsigned)m->g.nc, MG_MAX_N, 0, c->stream>>>(m->Y, in, m->g, out);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    return WCL_OK;
  }
  // `steps` minimal-residual steps on M x = b from x (x0 given: r = b - M x; else x = 0, r = b)
  wcl_status minres(float4* x, const float4* b, int steps, bool x0) {
    float4* r = fine(5);
    float4* ar = fine(6);
    const long n = nfine();
    if (x0) {
      WCL_CHECK(apply_M(ar, x));
      WCL_CHECK(copy((float2*)r, (const float2*)b, n));
      WCL_CHECK(axpby((float2*)r, (const float2*)ar, make_double2(-1, 0), make_double2(1, 0), n));
    } else {
      WCL_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * n, c->stream));
      WCL_CHECK(copy((float2*)r, (const float2*)b, n));
    }
    for (int s = 0; s < steps; s++) {
      WCL_CHECK(apply_M(ar, r));
      double2 den, num;
      WCL_CHECK(dot((const float2*)ar, (const float2*)ar, n, &den));
      if (!(den.x > 0)) break;
      WCL_CHECK(dot((const float2*)ar, (const float2*)r, n, &num));
      const double2 al = make_double2(num.x / den.x, num.y / den.x);
      WCL_CHECK(axpby((float2*)x, (const float2*)r, al, make_double2(1, 0), n));
      WCL_CHECK(axpby((float2*)r, (const float2*)ar, make_double2(-al.x, -al.y), make_double2(1, 0), n));
    }
    return WCL_OK;
  }
  // coarse GCR (restarted every nkrylov directions, modified Gram-Schmidt) on A_c x = b to a
  // relative tolerance or maxiter steps; x starts at zero
  wcl_status coarse_solve(float2* x, const float2* b, int* iters) {
    const long n = ncoarse();
    const int nk = std::max(1, std::min(m->prm.coarse_nkrylov, 64));
    float2* r = coarse(1);
    float2* Z = coarse(2);
    float2* W = coarse(2 + nk);
    WCL_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * n, c->stream));
    WCL_CHECK(copy(r, b, n));
    double2 bb;
    WCL_CHECK(dot(b, b, n, &bb));
    const double bnorm = std::sqrt(bb.x);
    *iters = 0;
    if (!(bnorm > 0)) return WCL_OK;
    double rn = bnorm;
    int k = 0;
    while (rn > m->prm.coarse_tol * bnorm && *iters < m->prm.coarse_maxiter) {
      if (k == nk) k = 0;
      float2* z = Z + (size_t)k * n;
      float2* w = W + (size_t)k * n;
      WCL_CHECK(copy(z, r, n));
      WCL_CHECK(coarse_apply(w, z));
      for (int j = 0; j < k; j++) {
        double2 be;
        WCL_CHECK(dot(W + (size_t)j * n, w, n, &be));
        WCL_CHECK(axpby(w, W + (size_t)j * n, make_double2(-be.x, -be.y), make_double2(1, 0), n));
        WCL_CHECK(axpby(z, Z + (size_t)j * n, make_double2(-be.x, -be.y), make_double2(1, 0), n));
      }
      double2 ww;
      WCL_CHECK(dot(w, w, n, &ww));
      if (!(ww.x > 0)) break;
      const double inv = 1.0 / std::sqrt(ww.x);
      WCL_CHECK(axpby(w, w, make_double2(0, 0), make_double2(inv, 0), n));
      WCL_CHECK(axpby(z, z, make_double2(0, 0), make_double2(inv, 0), n));
      double2 al;
      WCL_CHECK(dot(w, r, n, &al));
      WCL_CHECK(axpby(x, z, al, make_double2(1, 0), n));
      WCL_CHECK(axpby(r, w, make_double2(-al.x, -al.y), make_double2(1, 0), n));
      k++;
      (*iters)++;
      double2 rr;
      WCL_CHECK(dot(r, r, n, &rr));
      rn = std::sqrt(rr.x);
    }
    return WCL_OK;
  }
  // e = K-cycle(r)
  wcl_status cycle(float4* e, const float4* r, int* coarse_iters) {
    const long n = nfine();
    float4* r1 = fine(7);
    float4* t = fine(6);
    WCL_CHECK(minres(e, r, m->prm.pre, false));
    WCL_CHECK(apply_M(t, e));
    WCL_CHECK(copy((float2*)r1, (const float2*)r, n));
    WCL_CHECK(axpby((float2*)r1, (const float2*)t, make_double2(-1, 0), make_double2(1, 0), n));
    float2* rc = coarse(0);
    float2* ec = coarse(2 + 2 * std::max(1, std::min(m->prm.coarse_nkrylov, 64)));
    WCL_CHECK(restrict_(rc, r1));
    WCL_CHECK(coarse_solve(ec, rc, coarse_iters));
    WCL_CHECK(prolong(e, ec, true));
    if (m->prm.post > 0) WCL_CHECK(minres(e, r, m->prm.post, true));
    return WCL_OK;
  }
};

// The K-cycle on nr right-hand sides at once (batched layouts above): the same steps as
// Ctx::cycle, with the minimal-residual and Gram-Schmidt coefficients of every
// right-hand side computed and consumed on the device, and a fixed number of coarse GCR
// steps (coarse_maxiter; restarted every coarse_nkrylov), so nothing waits on the host.
struct BCtx {
  wcl_ctx* c;
  MgState* m;
  int nr;
  float4* in;   // the right-hand sides of the cycle
  float4* e;    // its result
  float4* rr;   // minimal-residual residual
  float4* ar;   // M rr
  float4* t;    // M e, then the fine residual restricted
  float2* cw;   // coarse: b, r, x, Z[nk], W[nk]
  double* part;
  float2* ca;
  float2* cb;
  int gb = 1;

  long half() const { return 6 * m->g.stride; }            // float4 in one parity of one RHS
  long pc() const { return 12 * m->g.stride; }              // complex numbers in one parity of one RHS
  long fine_c() const { return 2 * nr * pc(); }             // complex numbers of a whole batched field
  long ncv() const { return m->g.nc * m->g.n; }             // complex numbers of one coarse vector
  int nk() const { return std::max(1, std::min(m->prm.coarse_nkrylov, 64)); }
  float2* cvec(int k) const { return cw + (size_t)k * nr * ncv(); }

  wcl_status alloc(int nrhs) {
    nr = nrhs;
    const size_t fb = sizeof(float4) * 2 * nr * half();
    void* q;
    WCL_CHECK(ws_get(c, "mgb_fine", fb * 5, &q));
    in = static_cast<float4*>(q);
    e = in + 2 * nr * half();
    rr = e + 2 * nr * half();
    ar = rr + 2 * nr * half();
    t = ar + 2 * nr * half();
    WCL_CHECK(ws_get(c, "mgb_coarse", sizeof(float2) * nr * ncv() * (3 + 2 * nk()), &q));
    cw = static_cast<float2*>(q);
    gb = std::min(256, grid_of(2 * pc()));
    WCL_CHECK(ws_get(c, "mgb_part", sizeof(double) * 4 * nr * std::max(gb, 256), &q));
    part = static_cast<double*>(q);
    WCL_CHECK(ws_get(c, "mgb_coef", sizeof(float2) * 2 * nr, &q));
    ca = static_cast<float2*>(q);
    cb = ca + nr;
    return WCL_OK;
  }
  wcl_status apply_M(float4* out, const float4* x) {
    std::vector<wcl_ctx*> v{c};
    FieldRef ie{}, io{}, oe{}, oo{};
    ie.ptr[0] = const_cast<float4*>(x);
    io.ptr[0] = const_cast<float4*>(x) + nr * half();
    oe.ptr[0] = out;
    oo.ptr[0] = out + nr * half();
    WCL_CHECK(dslash(v, F32, nr, oe, io, &ie, 0, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, nullptr));
    WCL_CHECK(dslash(v, F32, nr, oo, ie, &io, 1, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, nullptr));
    return WCL_OK;
  }
  // coefficients of every right-hand side from <a, b> (and <a, cc>); fine: batched fine
  // fields (both parities), else coarse vectors
  wcl_status coef(const float2* a, const float2* b, const float2* cc, bool fine, int mode) {
    const long n = fine ? pc() : ncv();
    const long rs = fine ? pc() : ncv();
    const long seg2 = fine ? nr * pc() : 0;
    const int g = fine ? gb : std::min(64, grid_of(n));
    mgb_dot_kernel<<<dim3(g, nr), 256, 0, c->stream>>>(a, b, cc, n, rs, seg2, part);
    WCL_CUDA(cudaGetLastError());
    mgb_coef_kernel<<<1, 32 * ((nr + 31) / 32), 0, c->stream>>>(part, g, nr, mode, ca, cb);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    count_launch(c);
    return WCL_OK;
  }
  wcl_status axpy(float2* y, const float2* x, const float2* k, bool fine) {
    const long n = fine ? pc() : ncv();
    const long rs = n;
    const long seg2 = fine ? nr * pc() : 0;
    mgb_axpy_kernel<<<dim3(std::min(grid_of(fine ? 2 * n : n), 152 * 4), nr), 256, 0, c->stream>>>(y, x, k, n, rs, seg2);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    return WCL_OK;
  }
  // `steps` minimal-residual steps on M x = b from x (x0: r = b - M x; else x = 0, r = b)
  wcl_status minres(float4* x, const float4* b, int steps, bool x0) {
    const long n = fine_c();
    if (x0) {
      // rr = b - M x (mgb_rsub_kernel forms y = x - y in place)
      WCL_CHECK(apply_M(ar, x));
      WCL_CUDA(cudaMemcpyAsync(rr, ar, sizeof(float2) * n, cudaMemcpyDeviceToDevice, c->stream));
      mgb_rsub_kernel<<<grid_of(n), 256, 0, c->stream>>>((float2*)rr, (const float2*)b, n);
      WCL_CUDA(cudaGetLastError());
      count_launch(c);
    } else {
      WCL_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * n, c->stream));
      WCL_CUDA(cudaMemcpyAsync(rr, b, sizeof(float2) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    for (int s = 0; s < steps; s++) {
      WCL_CHECK(apply_M(ar, rr));
      WCL_CHECK(coef((const float2*)ar, (const float2*)ar, (const float2*)rr, true, MGB_MR));
      WCL_CHECK(axpy((float2*)x, (const float2*)rr, ca, true));
      WCL_CHECK(axpy((float2*)rr, (const float2*)ar, cb, true));
    }
    return WCL_OK;
  }
  // coarse GCR on A_c x = b from x = 0, a fixed number of steps
  wcl_status coarse_solve(float2* x, const float2* b, int steps) {
    const long n = (long)nr * ncv();
    float2* r = cvec(1);
    float2* Z = cvec(3);
    float2* W = cvec(3 + nk());
    WCL_CUDA(cudaMemsetAsync(x, 0, sizeof(float2) * n, c->stream));
    WCL_CUDA(cudaMemcpyAsync(r, b, sizeof(float2) * n, cudaMemcpyDeviceToDevice, c->stream));
    int k = 0;
    for (int it = 0; it < steps; it++) {
      if (k == nk()) k = 0;
      float2* z = Z + (size_t)k * nr * ncv();
      float2* w = W + (size_t)k * nr * ncv();
      WCL_CUDA(cudaMemcpyAsync(z, r, sizeof(float2) * n, cudaMemcpyDeviceToDevice, c->stream));
      mgb_coarse_apply_kernel<<<(unsigned)m->g.nc, MG_MAX_N, 0, c->stream>>>(m->Y, z, m->g, w, nr);
      WCL_CUDA(cudaGetLastError());
      count_launch(c);
      for (int j = 0; j < k; j++) {
        const float2* wj = W + (size_t)j * nr * ncv();
        const float2* zj = Z + (size_t)j * nr * ncv();
        WCL_CHECK(coef(wj, w, nullptr, false, MGB_PROJ));
        WCL_CHECK(axpy(w, wj, ca, false));
        WCL_CHECK(axpy(z, zj, ca, false));
      }
      WCL_CHECK(coef(w, w, nullptr, false, MGB_NORMINV));
      WCL_CHECK(axpy(w, nullptr, ca, false));
      WCL_CHECK(axpy(z, nullptr, ca, false));
      WCL_CHECK(coef(w, r, nullptr, false, MGB_COEF));
      WCL_CHECK(axpy(x, z, ca, false));
      WCL_CHECK(axpy(r, w, cb, false));
      k++;
    }
    return WCL_OK;
  }
  // e = K-cycle(in)
  wcl_status cycle() {
    const MgGeom& g = m->g;
    WCL_CHECK(minres(e, in, m->prm.pre, false));
    WCL_CHECK(apply_M(t, e));
    mgb_rsub_kernel<<<grid_of(fine_c()), 256, 0, c->stream>>>((float2*)t, (const float2*)in, fine_c());
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    float2* rc = cvec(0);
    float2* ec = cvec(2);
    const size_t sm = sizeof(float2) * g.bsites * 12 + sizeof(long) * g.bsites;
    mgb_restrict_kernel<<<(unsigned)(g.nc * nr), MGB_RG * MG_MAX_N, sm, c->stream>>>(t, m->P, g, rc, nr);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    WCL_CHECK(coarse_solve(ec, rc, std::max(1, m->prm.coarse_maxiter)));
    mgb_prolong_kernel<<<(unsigned)std::min((2 * g.stride + 127) / 128, 152L * 16), 128, 0, c->stream>>>(ec, m->P, g, e,
                                                                                                     nr);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    if (m->prm.post > 0) WCL_CHECK(minres(e, in, m->prm.post, true));
    return WCL_OK;
  }
};

// import a QDP complex128 full field (device or page-locked host) into a fine FP32 field
wcl_status import_full32(wcl_ctx* c, const void* src, float4* dst, long rhs_off_c) {
  std::vector<wcl_ctx*> v{c};
  FieldRef f64{};
  WCL_CHECK(ws_field(v, "mg_io64", F64, 2, &f64));  // even, odd
  const LatticeDevice& L = c->lat;
  const long rs = 2 * L.vh * 12;
  WCL_CUDA(import_fermion(L, static_cast<const double2*>(src) + rhs_off_c, rs, 0, 1, f64.ptr[0], c->d_flags,
                          c->stream));
  WCL_CUDA(import_fermion(L, static_cast<const double2*>(src) + rhs_off_c, rs, L.vh * 12, 1,
                          static_cast<double2*>(f64.ptr[0]) + 12 * L.stride, c->d_flags, c->stream));
  count_launch(c);
  count_launch(c);
  mg_to32_kernel<<<grid_of(12 * L.stride), 256, 0, c->stream>>>(static_cast<const double2*>(f64.ptr[0]), dst,
                                                                L.stride);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  return WCL_OK;
}

wcl_status export_full32(wcl_ctx* c, const float4* src, void* dst) {
  std::vector<wcl_ctx*> v{c};
  FieldRef f64{};
  WCL_CHECK(ws_field(v, "mg_io64", F64, 2, &f64));
  const LatticeDevice& L = c->lat;
  WCL_CUDA(cudaMemsetAsync(f64.ptr[0], 0, sizeof(double2) * 24 * L.stride, c->stream));
  mg_add32into64_kernel<<<grid_of(12 * L.stride), 256, 0, c->stream>>>(static_cast<double2*>(f64.ptr[0]), src,
                                                                       L.stride);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  const long rs = 2 * L.vh * 12;
  WCL_CUDA(export_fermion(L, f64.ptr[0], 1, dst, rs, 0, c->stream));
  WCL_CUDA(export_fermion(L, static_cast<double2*>(f64.ptr[0]) + 12 * L.stride, 1, dst, rs, L.vh * 12, c->stream));
  count_launch(c);
  count_launch(c);
  return WCL_OK;
}

wcl_status check_ready(wcl_ctx* c, const char* what) {
  if (!c) return WCL_ERR_INVALID_ARG;
  if (!c->lat.loaded) {
    set_error("%s: no gauge field loaded", what);
    return WCL_ERR_NO_GAUGE;
  }
  if (!mg_of(c) || !mg_of(c)->ready) {
    set_error("%s: no multigrid hierarchy (wcl_mg_setup)", what);
    return WCL_ERR_NO_PRECOND;
  }
  return WCL_OK;
}

}  // namespace

// z_e = [K(r_e (+) 0)]_e for nrhs even-site FP32 fields (the library's nrhs parity-field
// layout, consecutive right-hand sides): the batched K-cycle of the whole-lattice M
// applied to the residual embedded with zero odd sites.  Since the even-even block of
// M^-1 is M_hat^-1, this preconditions flexible GCR on M_hat (WCL_FGCR_MG_BATCHED).
wcl_status mg_batched_cycle(wcl_ctx* c, int nrhs, const void* r_even, void* z_even) {
  WCL_CHECK(check_ready(c, "batched multigrid cycle"));
  BCtx b{c, mg_of(c)};
  WCL_CHECK(b.alloc(nrhs));
  const size_t pb = sizeof(float4) * nrhs * b.half();
  WCL_CUDA(cudaMemcpyAsync(b.in, r_even, pb, cudaMemcpyDeviceToDevice, c->stream));
  WCL_CUDA(cudaMemsetAsync(b.in + nrhs * b.half(), 0, pb, c->stream));
  WCL_CHECK(b.cycle());
  WCL_CUDA(cudaMemcpyAsync(z_even, b.e, pb, cudaMemcpyDeviceToDevice, c->stream));
  return WCL_OK;
}

// the flexible-GCR solve of M x = b, one right-hand side, preconditioned by the K-cycle,
// in FP32 between FP64 true-residual restarts (used by wcl_invert with WCL_FGCR_MG)
wcl_status mg_solve_one(wcl_ctx* c, const void* d_b, void* d_x, long rhs_off_c, const wcl_solve_params& prm,
                        wcl_solve_info* info) {
  WCL_CHECK(check_ready(c, "wcl_invert (multigrid)"));
  MgState* m = mg_of(c);
  Ctx k{c, m};
  std::vector<wcl_ctx*> v{c};
  const LatticeDevice& L = c->lat;
  const long n = k.nfine();
  const long n64 = 24 * L.stride;  // complex numbers of a full FP64 field
  FieldRef b64{}, x64{}, r64{}, y64{};
  WCL_CHECK(ws_field(v, "mg_b64", F64, 2, &b64));
  WCL_CHECK(ws_field(v, "mg_x64", F64, 2, &x64));
  WCL_CHECK(ws_field(v, "mg_r64", F64, 2, &r64));
  WCL_CHECK(ws_field(v, "mg_y64", F64, 2, &y64));
  const int nk = std::max(1, std::min(prm.gcr_nkrylov, 64));
  void* q;
  WCL_CHECK(ws_get(c, "mg_gcr", sizeof(float4) * 2 * 6 * L.stride * (2 * nk + 2), &q));
  float4* Zs = static_cast<float4*>(q);
  float4* Ws = Zs + (size_t)nk * 2 * 6 * L.stride;
  float4* x32 = Ws + (size_t)nk * 2 * 6 * L.stride;
  float4* r32 = x32 + 2 * 6 * L.stride;
  const long rs = 2 * L.vh * 12;
  double2* b64p = static_cast<double2*>(b64.ptr[0]);
  double2* x64p = static_cast<double2*>(x64.ptr[0]);
  double2* r64p = static_cast<double2*>(r64.ptr[0]);
  double2* y64p = static_cast<double2*>(y64.ptr[0]);
  WCL_CUDA(import_fermion(L, static_cast<const double2*>(d_b) + rhs_off_c, rs, 0, 1, b64p, c->d_flags, c->stream));
  WCL_CUDA(import_fermion(L, static_cast<const double2*>(d_b) + rhs_off_c, rs, L.vh * 12, 1, b64p + 12 * L.stride,
                          c->d_flags, c->stream));
  count_launch(c);
  count_launch(c);
  WCL_CUDA(cudaMemsetAsync(x64p, 0, sizeof(double2) * n64, c->stream));
  WCL_CUDA(cudaMemcpyAsync(r64p, b64p, sizeof(double2) * n64, cudaMemcpyDeviceToDevice, c->stream));
  auto norm64 = [&](const double2* a, double* out) -> wcl_status {
    const int gb = std::min(MG_PART, grid_of(n64));
    mg_norm64_kernel<<<gb, 256, 0, c->stream>>>(a, n64, m->part);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    WCL_CUDA(cudaMemcpyAsync(m->hpart.data(), m->part, sizeof(double) * gb, cudaMemcpyDeviceToHost, c->stream));
    WCL_CUDA(cudaStreamSynchronize(c->stream));
    double s = 0;
    for (int j = 0; j < gb; j++) s += m->hpart[j];
    *out = s;
    return WCL_OK;
  };
  double b2;
  WCL_CHECK(norm64(b64p, &b2));
  info->iters = 0;
  info->reliable_updates = 0;
  info->status = WCL_OK;
  info->true_residual = 0;
  if (!(b2 > 0)) {
    WCL_CUDA(cudaMemsetAsync(x64p, 0, sizeof(double2) * n64, c->stream));
  } else {
    double r2 = b2;
    const double tol = prm.tol;
    int restarts = 0;
    while (std::sqrt(r2 / b2) > tol) {
      if (info->iters >= prm.maxiter || restarts > 50) {
        info->status = WCL_ERR_NOT_CONVERGED;
        break;
      }
      // inner FP32 FGCR on M e = r (relative target: what the FP64 residual still needs)
      mg_to32_kernel<<<grid_of(12 * L.stride), 256, 0, c->stream>>>(r64p, r32, L.stride);
      WCL_CUDA(cudaGetLastError());
      count_launch(c);
      WCL_CUDA(cudaMemsetAsync(x32, 0, sizeof(float2) * n, c->stream));
      const double rnorm0 = std::sqrt(r2);
      const double target = std::max(0.5 * tol * std::sqrt(b2) / rnorm0, 1e-6);
      double rn = rnorm0;
      int kk = 0;
      while (rn > target * rnorm0 && info->iters < prm.maxiter) {
        if (kk == nk) kk = 0;
        float4* z = Zs + (size_t)kk * 2 * 6 * L.stride;
        float4* w = Ws + (size_t)kk * 2 * 6 * L.stride;
        int ci = 0;
        WCL_CHECK(k.cycle(z, r32, &ci));
        WCL_CHECK(k.apply_M(w, z));
        for (int j = 0; j < kk; j++) {
          const float2* wj = (const float2*)(Ws + (size_t)j * 2 * 6 * L.stride);
          const float2* zj = (const float2*)(Zs + (size_t)j * 2 * 6 * L.stride);
          double2 be;
          WCL_CHECK(k.dot(wj, (const float2*)w, n, &be));
          WCL_CHECK(k.axpby((float2*)w, wj, make_double2(-be.x, -be.y), make_double2(1, 0), n));
          WCL_CHECK(k.axpby((float2*)z, zj, make_double2(-be.x, -be.y), make_double2(1, 0), n));
        }
        double2 ww;
        WCL_CHECK(k.dot((const float2*)w, (const float2*)w, n, &ww));
        if (!(ww.x > 0)) break;
        const double inv = 1.0 / std::sqrt(ww.x);
        WCL_CHECK(k.axpby((float2*)w, (const float2*)w, make_double2(0, 0), make_double2(inv, 0), n));
        WCL_CHECK(k.axpby((float2*)z, (const float2*)z, make_double2(0, 0), make_double2(inv, 0), n));
        double2 al;
        WCL_CHECK(k.dot((const float2*)w, (const float2*)r32, n, &al));
        WCL_CHECK(k.axpby((float2*)x32, (const float2*)z, al, make_double2(1, 0), n));
        WCL_CHECK(k.axpby((float2*)r32, (const float2*)w, make_double2(-al.x, -al.y), make_double2(1, 0), n));
        kk++;
        info->iters++;
        double2 rr;
        WCL_CHECK(k.dot((const float2*)r32, (const float2*)r32, n, &rr));
        rn = std::sqrt(rr.x);
        if (!(rn == rn)) break;
      }
      // x += e; r = b - M x in FP64 (the true residual of the whole system)
      mg_add32into64_kernel<<<grid_of(12 * L.stride), 256, 0, c->stream>>>(x64p, x32, L.stride);
      WCL_CUDA(cudaGetLastError());
      count_launch(c);
      FieldRef xe{}, xo{}, ye{}, yo{};
      xe.ptr[0] = x64p;
      xo.ptr[0] = x64p + 12 * L.stride;
      ye.ptr[0] = y64p;
      yo.ptr[0] = y64p + 12 * L.stride;
      WCL_CHECK(dslash(v, F64, 1, ye, xo, &xe, 0, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, nullptr));
      WCL_CHECK(dslash(v, F64, 1, yo, xe, &xo, 1, false, CL_NONE, CL_A, C_MKAPPA, C_ONE, nullptr));
      mg_sub64_kernel<<<grid_of(n64), 256, 0, c->stream>>>(r64p, b64p, y64p, n64);
      WCL_CUDA(cudaGetLastError());
      count_launch(c);
      WCL_CHECK(norm64(r64p, &r2));
      restarts++;
      info->reliable_updates++;
      if (!(r2 == r2)) {
        info->status = WCL_ERR_NONFINITE;
        break;
      }
    }
    info->true_residual = std::sqrt(r2 / b2);
  }
  WCL_CUDA(export_fermion(L, x64p, 1, static_cast<double2*>(d_x) + rhs_off_c, rs, 0, c->stream));
  WCL_CUDA(export_fermion(L, x64p + 12 * L.stride, 1, static_cast<double2*>(d_x) + rhs_off_c, rs, L.vh * 12,
                          c->stream));
  count_launch(c);
  count_launch(c);
  if (info->status == WCL_OK && !(info->true_residual <= prm.tol)) info->status = WCL_ERR_NOT_CONVERGED;
  return WCL_OK;
}

}  // namespace wcl

using namespace wcl;

extern "C" {

void wcl_default_mg_params(wcl_mg_params* p) {
  if (!p) return;
  for (int d = 0; d < 4; d++) p->block[d] = 4;
  p->nvec = 24;
  p->relax_steps = 20;
  p->pre = 2;
  p->post = 2;
  p->coarse_tol = 0.1;
  p->coarse_maxiter = 50;
  p->coarse_nkrylov = 8;
}

wcl_status wcl_mg_setup(wcl_ctx* c, const void* d_starts, const wcl_mg_params* prm) {
  if (!c || !d_starts || !prm) {
    set_error("wcl_mg_setup: null pointer");
    return WCL_ERR_INVALID_ARG;
  }
  if (!c->lat.loaded) {
    set_error("wcl_mg_setup: no gauge field loaded");
    return WCL_ERR_NO_GAUGE;
  }
  MgGeom g{};
  for (int d = 0; d < 4; d++) {
    g.dims[d] = c->lat.dims[d];
    g.block[d] = prm->block[d];
    if (prm->block[d] < 1 || c->lat.dims[d] % prm->block[d]) {
      set_error("wcl_mg_setup: block %d does not divide extent %d of direction %d", prm->block[d], c->lat.dims[d], d);
      return WCL_ERR_INVALID_ARG;
    }
    g.cdims[d] = c->lat.dims[d] / prm->block[d];
  }
  g.lxh = g.dims[0] / 2;
  g.stride = c->lat.stride;
  g.bsites = prm->block[0] * prm->block[1] * prm->block[2] * prm->block[3];
  g.nc = (long)g.cdims[0] * g.cdims[1] * g.cdims[2] * g.cdims[3];
  g.nv = prm->nvec;
  g.n = 2 * prm->nvec;
  if (prm->nvec < 1 || prm->nvec > MG_MAX_NV || prm->nvec > g.bsites * 6 || prm->relax_steps < 0 || prm->pre < 0 ||
      prm->post < 0 || prm->coarse_maxiter < 0 || prm->coarse_nkrylov < 1 || prm->coarse_nkrylov > 64 ||
      !(prm->coarse_tol >= 0)) {
    set_error("wcl_mg_setup: invalid parameters (1 <= nvec <= min(%d, 6 x block sites), steps >= 0, "
              "1 <= coarse_nkrylov <= 64)", MG_MAX_NV);
    return WCL_ERR_INVALID_ARG;
  }
  const void* starts = nullptr;
  if (!wcl_resolve_field(c, d_starts, &starts, "wcl_mg_setup starts")) return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  mg_free(c);
  MgState* m = new (std::nothrow) MgState;
  if (!m) return wcl_leave(c, WCL_ERR_OOM);
  c->mg = m;
  m->g = g;
  m->prm = *prm;
  m->hpart.assign(2 * MG_PART, 0.0);
  const int nk = std::max(1, std::min(prm->coarse_nkrylov, 64));
  cudaError_t e = cudaMalloc(&m->P, sizeof(float2) * 2 * g.stride * 12 * g.nv);
  if (e == cudaSuccess) e = cudaMalloc(&m->Y, sizeof(float2) * 9 * g.nc * g.n * g.n);
  if (e == cudaSuccess) e = cudaMalloc(&m->cw, sizeof(float2) * (size_t)(3 + 2 * nk) * g.nc * g.n);
  if (e == cudaSuccess) e = cudaMalloc(&m->fw, sizeof(float4) * (size_t)MG_FINE * 2 * 6 * g.stride);
  if (e == cudaSuccess) e = cudaMalloc(&m->part, sizeof(double) * 2 * MG_PART);
  if (e != cudaSuccess) {
    mg_free(c);
    return wcl_leave(c, cuda_fail(e, "wcl_mg_setup: allocation"));
  }
  e = cudaMemsetAsync(m->P, 0, sizeof(float2) * 2 * g.stride * 12 * g.nv, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->fw, 0, sizeof(float4) * (size_t)MG_FINE * 2 * 6 * g.stride, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return wcl_leave(c, cuda_fail(e, "wcl_mg_setup: clear"));
  Ctx k{c, m};
  const long n = k.nfine();
  const long vol_c = 2 * c->lat.vh * 12;  // complex numbers of one QDP fermion
  // null space: relax each start towards M x = 0, normalise, copy into column j of P
  for (int j = 0; j < g.nv; j++) {
    float4* x = k.fine(0);
    float4* zero = k.fine(1);
    wcl_status s = import_full32(c, starts, x, (long)j * vol_c);
    if (s == WCL_OK) s = k.minres(x, zero, prm->relax_steps, true);  // fine(1) stays zero: b = 0
    double2 nn{};
    if (s == WCL_OK) s = k.dot((const float2*)x, (const float2*)x, n, &nn);
    if (s == WCL_OK && !(nn.x > 0)) {
      set_error("wcl_mg_setup: null vector %d vanished", j);
      s = WCL_ERR_BREAKDOWN;
    }
    if (s == WCL_OK) s = k.axpby((float2*)x, (const float2*)x, make_double2(0, 0), make_double2(1.0 / std::sqrt(nn.x), 0), n);
    if (s == WCL_OK) {
      mg_fill_kernel<<<grid_of(2 * g.stride * 12), 256, 0, c->stream>>>(x, j, g, m->P);
      e = cudaGetLastError();
      if (e != cudaSuccess) s = cuda_fail(e, "mg_fill_kernel");
      count_launch(c);
    }
    if (s != WCL_OK) {
      mg_free(c);
      return wcl_leave(c, s);
    }
  }
  mg_orthonormalize_kernel<<<(unsigned)(2 * g.nc), 256, 0, c->stream>>>(m->P, g, c->d_flags);
  e = cudaGetLastError();
  count_launch(c);
  // coarse operator from the links, the clover term and P
  MgBuildArgs a{};
  a.g = g;
  for (int p = 0; p < 2; p++) {
    a.gauge[p] = c->lat.gauge[F32][p];
    a.clov[p] = c->lat.clov[F32][p];
  }
  a.kappa = c->lat.kappa;
  a.tw_f = (float)c->lat.tw;
  a.tbw_f = (float)((double)c->lat.tb * c->lat.tw);
  a.P = m->P;
  a.Y = m->Y;
  const size_t sm = sizeof(float2) * 24 * g.n;
  if (e == cudaSuccess) {
    mg_build_kernel<<<(unsigned)(9 * g.nc), MG_BUILD_THREADS, sm, c->stream>>>(a);
    e = cudaGetLastError();
    count_launch(c);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    mg_free(c);
    return wcl_leave(c, cuda_fail(e, "wcl_mg_setup"));
  }
  if (*c->h_flags & 9) {
    set_error("wcl_mg_setup: %s", (*c->h_flags & 1) ? "non-finite start vector" : "null vectors linearly dependent in a block");
    mg_free(c);
    return wcl_leave(c, (*c->h_flags & 1) ? WCL_ERR_NONFINITE : WCL_ERR_BREAKDOWN);
  }
  m->ready = true;
  return wcl_leave(c, WCL_OK);
}

wcl_status wcl_mg_cycle(wcl_ctx* c, void* d_out, const void* d_in, int* coarse_iters) {
  WCL_CHECK(check_ready(c, "wcl_mg_cycle"));
  if (!d_out || !d_in) return WCL_ERR_INVALID_ARG;
  const void* in = nullptr;
  const void* outc = nullptr;
  if (!wcl_resolve_field(c, d_in, &in, "wcl_mg_cycle d_in") ||
      !wcl_resolve_field(c, d_out, &outc, "wcl_mg_cycle d_out"))
    return WCL_ERR_INVALID_ARG;
  void* out = const_cast<void*>(outc);
  WCL_CHECK(wcl_enter(c));
  Ctx k{c, mg_of(c)};
  int ci = 0;
  wcl_status s = import_full32(c, in, k.fine(3), 0);
  if (s == WCL_OK) s = k.cycle(k.fine(4), k.fine(3), &ci);
  if (s == WCL_OK) s = export_full32(c, k.fine(4), out);
  if (coarse_iters) *coarse_iters = ci;
  return wcl_leave(c, s);
}

wcl_status wcl_mg_cycle_batched(wcl_ctx* c, void* d_out, const void* d_in, int nrhs) {
  if (!c || !d_out || !d_in || nrhs < 1 || nrhs > 12) {
    set_error("wcl_mg_cycle_batched: invalid argument (1 <= nrhs <= 12)");
    return WCL_ERR_INVALID_ARG;
  }
  WCL_CHECK(check_ready(c, "wcl_mg_cycle_batched"));
  const void* in = nullptr;
  const void* outc = nullptr;
  if (!wcl_resolve_field(c, d_in, &in, "wcl_mg_cycle_batched in") ||
      !wcl_resolve_field(c, d_out, &outc, "wcl_mg_cycle_batched out"))
    return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  BCtx b{c, mg_of(c)};
  WCL_CHECK(b.alloc(nrhs));
  Ctx k{c, mg_of(c)};
  float4* tmp = k.fine(0);  // one whole-lattice FP32 field: [even 6 x stride][odd 6 x stride]
  const long h = b.half();
  const long rs = 2 * c->lat.vh * 12;
  for (int r = 0; r < nrhs; r++) {
    WCL_CHECK(import_full32(c, static_cast<const double2*>(in) + (long)r * rs, tmp, 0));
    WCL_CUDA(cudaMemcpyAsync(b.in + r * h, tmp, sizeof(float4) * h, cudaMemcpyDeviceToDevice, c->stream));
    WCL_CUDA(cudaMemcpyAsync(b.in + (nrhs + r) * h, tmp + h, sizeof(float4) * h, cudaMemcpyDeviceToDevice,
                             c->stream));
  }
  WCL_CHECK(b.cycle());
  for (int r = 0; r < nrhs; r++) {
    WCL_CUDA(cudaMemcpyAsync(tmp, b.e + r * h, sizeof(float4) * h, cudaMemcpyDeviceToDevice, c->stream));
    WCL_CUDA(cudaMemcpyAsync(tmp + h, b.e + (nrhs + r) * h, sizeof(float4) * h, cudaMemcpyDeviceToDevice,
                             c->stream));
    WCL_CHECK(export_full32(c, tmp, static_cast<double2*>(const_cast<void*>(outc)) + (long)r * rs));
  }
  return wcl_leave(c, WCL_OK);
}

wcl_status wcl_mg_restrict(wcl_ctx* c, void* d_coarse, const void* d_fine) {
  WCL_CHECK(check_ready(c, "wcl_mg_restrict"));
  if (!d_coarse || !d_fine) return WCL_ERR_INVALID_ARG;
  const void* in = nullptr;
  if (!wcl_resolve_field(c, d_fine, &in, "wcl_mg_restrict d_fine")) return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  Ctx k{c, mg_of(c)};
  const long nc = k.ncoarse();
  wcl_status s = import_full32(c, in, k.fine(3), 0);
  if (s == WCL_OK) s = k.restrict_(k.coarse(0), k.fine(3));
  if (s == WCL_OK) {
    // coarse vector out as complex128
    std::vector<float2> h(nc);
    cudaError_t e = cudaMemcpyAsync(h.data(), k.coarse(0), sizeof(float2) * nc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    std::vector<double2> d(nc);
    for (long q = 0; q < nc; q++) d[q] = make_double2(h[q].x, h[q].y);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_coarse, d.data(), sizeof(double2) * nc, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "wcl_mg_restrict copy");
  }
  return wcl_leave(c, s);
}

static wcl_status coarse_in(wcl_ctx* c, const void* d_coarse, float2* dst, long nc) {
  std::vector<double2> d(nc);
  cudaError_t e = cudaMemcpyAsync(d.data(), d_coarse, sizeof(double2) * nc, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "coarse vector copy");
  std::vector<float2> h(nc);
  for (long q = 0; q < nc; q++) h[q] = make_float2((float)d[q].x, (float)d[q].y);
  e = cudaMemcpyAsync(dst, h.data(), sizeof(float2) * nc, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "coarse vector copy");
  return WCL_OK;
}

wcl_status wcl_mg_prolong(wcl_ctx* c, void* d_fine, const void* d_coarse) {
  WCL_CHECK(check_ready(c, "wcl_mg_prolong"));
  if (!d_coarse || !d_fine) return WCL_ERR_INVALID_ARG;
  const void* outc = nullptr;
  if (!wcl_resolve_field(c, d_fine, &outc, "wcl_mg_prolong d_fine")) return WCL_ERR_INVALID_ARG;
  void* out = const_cast<void*>(outc);
  WCL_CHECK(wcl_enter(c));
  Ctx k{c, mg_of(c)};
  wcl_status s = coarse_in(c, d_coarse, k.coarse(0), k.ncoarse());
  if (s == WCL_OK) s = k.prolong(k.fine(3), k.coarse(0), false);
  if (s == WCL_OK) s = export_full32(c, k.fine(3), out);
  return wcl_leave(c, s);
}

wcl_status wcl_mg_coarse_apply(wcl_ctx* c, void* d_out, const void* d_in) {
  WCL_CHECK(check_ready(c, "wcl_mg_coarse_apply"));
  if (!d_out || !d_in) return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  Ctx k{c, mg_of(c)};
  const long nc = k.ncoarse();
  wcl_status s = coarse_in(c, d_in, k.coarse(0), nc);
  if (s == WCL_OK) s = k.coarse_apply(k.coarse(1), k.coarse(0));
  if (s == WCL_OK) {
    std::vector<float2> h(nc);
    cudaError_t e = cudaMemcpyAsync(h.data(), k.coarse(1), sizeof(float2) * nc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    std::vector<double2> d(nc);
    for (long q = 0; q < nc; q++) d[q] = make_double2(h[q].x, h[q].y);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_out, d.data(), sizeof(double2) * nc, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) s = cuda_fail(e, "wcl_mg_coarse_apply copy");
  }
  return wcl_leave(c, s);
}

wcl_status wcl_mg_get_prolongator(wcl_ctx* c, double* h_P) {
  WCL_CHECK(check_ready(c, "wcl_mg_get_prolongator"));
  if (!h_P) return WCL_ERR_INVALID_ARG;
  MgState* m = mg_of(c);
  const MgGeom& g = m->g;
  WCL_CHECK(wcl_enter(c));
  std::vector<float2> h((size_t)2 * g.stride * 12 * g.nv);
  cudaError_t e = cudaMemcpyAsync(h.data(), m->P, sizeof(float2) * h.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return wcl_leave(c, cuda_fail(e, "wcl_mg_get_prolongator"));
  // out: QDP site order [2][Lt][Lz][Ly][Lx/2], then [12][2 nv] (row m = 3 spin + colour,
  // column chi nv + k; zero where the chirality of m and of the column differ)
  const long vh = c->lat.vh;
  for (int p = 0; p < 2; p++)
    for (long i = 0; i < vh; i++)
      for (int mm = 0; mm < 12; mm++)
        for (int j = 0; j < g.n; j++) {
          const long o = ((((long)p * vh + i) * 12 + mm) * g.n + j) * 2;
          float2 v = make_float2(0.f, 0.f);
          if (mm / 6 == j / g.nv) v = h[((size_t)(p * g.stride + i) * 12 + mm) * g.nv + j % g.nv];
          h_P[o] = v.x;
          h_P[o + 1] = v.y;
        }
  return wcl_leave(c, WCL_OK);
}

wcl_status wcl_mg_get_stencil(wcl_ctx* c, double* h_Y) {
  WCL_CHECK(check_ready(c, "wcl_mg_get_stencil"));
  if (!h_Y) return WCL_ERR_INVALID_ARG;
  MgState* m = mg_of(c);
  const MgGeom& g = m->g;
  WCL_CHECK(wcl_enter(c));
  std::vector<float2> h((size_t)9 * g.nc * g.n * g.n);
  cudaError_t e = cudaMemcpyAsync(h.data(), m->Y, sizeof(float2) * h.size(), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return wcl_leave(c, cuda_fail(e, "wcl_mg_get_stencil"));
  // out: [9][coarse site][row a][column b] complex128 (device storage is column-major)
  for (long q = 0; q < 9 * g.nc; q++)
    for (int ra = 0; ra < g.n; ra++)
      for (int cb = 0; cb < g.n; cb++) {
        const float2 v = h[(size_t)q * g.n * g.n + (size_t)cb * g.n + ra];
        const size_t o = ((size_t)q * g.n * g.n + (size_t)ra * g.n + cb) * 2;
        h_Y[o] = v.x;
        h_Y[o + 1] = v.y;
      }
  return wcl_leave(c, WCL_OK);
}

}  // extern "C"
