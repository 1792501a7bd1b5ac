// Gauge import (QDP complex128 -> 12-real links in every precision, with the
// SU(3) check that 12-real storage relies on), clover construction and
// inversion in FP64 (Eq. 5 clover term, built at gauge load as in Sec. III.B),
// and fermion import/export between the QDP layout and the internal layout.
#include "fields.cuh"

namespace wcl {

// ---------------------------------------------------------------------------
// QDP index helpers: gauge [4][2][vh][3][3], fermion [2][vh][4][3] (complex)
struct QdpGeom {
  int Lx, Ly, Lz, Lt, lxh;
  long vh;
};

__device__ __forceinline__ long cb_index(const QdpGeom& q, int x, int y, int z, int t) {
  return (((long)t * q.Lz + z) * q.Ly + y) * q.lxh + (x >> 1);
}

__device__ __forceinline__ void site_coords(const QdpGeom& q, int p, long i, int& x, int& y, int& z, int& t) {
  const int xh = (int)(i % q.lxh);
  int rem = (int)(i / q.lxh);
  y = rem % q.Ly;
  rem /= q.Ly;
  z = rem % q.Lz;
  t = rem / q.Lz;
  x = 2 * xh + ((p + y + z + t) & 1);
}

// ---------------------------------------------------------------------------
// gauge import: check + pack rows 0, 1 of every link into the four precisions
struct GaugePack {
  void* g64[2];
  void* g32[2];
  void* g16[2];
  void* gb16[2];
  long stride;
};

__global__ void gauge_import_kernel(const double2* __restrict__ qdp, QdpGeom q, GaugePack out, double tol,
                                    int* __restrict__ flags) {
  const long n = 8 * q.vh;  // (mu, parity) pairs x sites
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const long i = idx % q.vh;
    const int mp = (int)(idx / q.vh);
    const int mu = mp >> 1, p = mp & 1;
    const double2* src = qdp + ((long)(mu * 2 + p) * q.vh + i) * 9;
    cpx<double> u[3][3];
    bool finite = true;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double2 v = src[3 * a + b];
        u[a][b] = {v.x, v.y};
        finite = finite && isfinite(v.x) && isfinite(v.y);
      }
    if (!finite) {
      atomicOr(flags, 1);
      continue;
    }
    // unitarity and determinant
    double dev = 0.0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        cpx<double> s = {0, 0};
        for (int c = 0; c < 3; c++) cfma_conj(s, u[b][c], u[a][c]);  // (U U^+)_{ab} = sum_c U_ac conj(U_bc)
        s.re -= (a == b) ? 1.0 : 0.0;
        dev = fmax(dev, fmax(fabs(s.re), fabs(s.im)));
      }
    cpx<double> det = u[0][0] * (u[1][1] * u[2][2] - u[1][2] * u[2][1]) -
                      u[0][1] * (u[1][0] * u[2][2] - u[1][2] * u[2][0]) +
                      u[0][2] * (u[1][0] * u[2][1] - u[1][1] * u[2][0]);
    dev = fmax(dev, fmax(fabs(det.re - 1.0), fabs(det.im)));
    if (!(dev <= tol)) atomicOr(flags, 2);
    const long st = out.stride;
    // F64: all 9 entries as double2 chunks
    double2* d64 = static_cast<double2*>(out.g64[p]) + (long)mu * 9 * st;
    for (int k = 0; k < 9; k++) d64[k * st + i] = make_double2(u[k / 3][k % 3].re, u[k / 3][k % 3].im);
    // F32: 3 float4 chunks
    float4* d32 = static_cast<float4*>(out.g32[p]) + (long)mu * 3 * st;
    for (int k = 0; k < 3; k++) {
      cpx<double> a0 = u[(2 * k) / 3][(2 * k) % 3], a1 = u[(2 * k + 1) / 3][(2 * k + 1) % 3];
      d32[k * st + i] = make_float4((float)a0.re, (float)a0.im, (float)a1.re, (float)a1.im);
    }
    // F16 / BF16: 3 uint2 chunks (entries of a unitary matrix are bounded by 1)
    uint2* d16 = static_cast<uint2*>(out.g16[p]) + (long)mu * 3 * st;
    uint2* db16 = static_cast<uint2*>(out.gb16[p]) + (long)mu * 3 * st;
    for (int k = 0; k < 3; k++) {
      cpx<double> a0 = u[(2 * k) / 3][(2 * k) % 3], a1 = u[(2 * k + 1) / 3][(2 * k + 1) % 3];
      d16[k * st + i] = make_uint2(pack2<F16>((float)a0.re, (float)a0.im), pack2<F16>((float)a1.re, (float)a1.im));
      db16[k * st + i] = make_uint2(pack2<BF16>((float)a0.re, (float)a0.im), pack2<BF16>((float)a1.re, (float)a1.im));
    }
  }
}

// ---------------------------------------------------------------------------
// clover build: F_{mu nu} from the four leaves, A = 1 - kappa csw sum sigma F,
// per chiral 6x6 block; inverse by Gauss-Jordan with partial pivoting (FP64).

// DeGrand-Rossi gamma_mu, mu = x, y, z, t, as (re, im) 4x4
__constant__ double c_gamma[4][4][4][2] = {
    {{{0, 0}, {0, 0}, {0, 0}, {0, 1}}, {{0, 0}, {0, 0}, {0, 1}, {0, 0}}, {{0, 0}, {0, -1}, {0, 0}, {0, 0}}, {{0, -1}, {0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 0}, {-1, 0}}, {{0, 0}, {0, 0}, {1, 0}, {0, 0}}, {{0, 0}, {1, 0}, {0, 0}, {0, 0}}, {{-1, 0}, {0, 0}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {0, 1}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {0, -1}}, {{0, -1}, {0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {0, 1}, {0, 0}, {0, 0}}},
    {{{0, 0}, {0, 0}, {1, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {1, 0}}, {{1, 0}, {0, 0}, {0, 0}, {0, 0}}, {{0, 0}, {1, 0}, {0, 0}, {0, 0}}}};

struct Mat3 {
  cpx<double> m[3][3];
};

__device__ __forceinline__ Mat3 mul(const Mat3& a, const Mat3& b) {
  Mat3 c;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cpx<double> s = {0, 0};
      for (int k = 0; k < 3; k++) cfma(s, a.m[i][k], b.m[k][j]);
      c.m[i][j] = s;
    }
  return c;
}
__device__ __forceinline__ Mat3 dag(const Mat3& a) {
  Mat3 c;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) c.m[i][j] = conj(a.m[j][i]);
  return c;
}

__device__ Mat3 load_link(const double2* qdp, const QdpGeom& q, int mu, int x, int y, int z, int t) {
  x = (x + q.Lx) % q.Lx;
  y = (y + q.Ly) % q.Ly;
  z = (z + q.Lz) % q.Lz;
  t = (t + q.Lt) % q.Lt;
  const int p = (x + y + z + t) & 1;
  const double2* src = qdp + ((long)(mu * 2 + p) * q.vh + cb_index(q, x, y, z, t)) * 9;
  Mat3 u;
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      double2 v = src[3 * a + b];
      u.m[a][b] = {v.x, v.y};
    }
  return u;
}

__device__ void field_strength(const double2* qdp, const QdpGeom& q, int mu, int nu, const int c[4], Mat3& F) {
  auto L = [&](int d, int dm, int dn) {
    int cc[4] = {c[0], c[1], c[2], c[3]};
    cc[mu] += dm;
    cc[nu] += dn;
    return load_link(qdp, q, d, cc[0], cc[1], cc[2], cc[3]);
  };
  // leaves with orientation +mu, +nu, -mu, -nu starting at s
  Mat3 l1 = mul(mul(L(mu, 0, 0), L(nu, 1, 0)), mul(dag(L(mu, 0, 1)), dag(L(nu, 0, 0))));
  Mat3 l2 = mul(mul(L(nu, 0, 0), dag(L(mu, -1, 1))), mul(dag(L(nu, -1, 0)), L(mu, -1, 0)));
  Mat3 l3 = mul(mul(dag(L(mu, -1, 0)), dag(L(nu, -1, -1))), mul(L(mu, -1, -1), L(nu, 0, -1)));
  Mat3 l4 = mul(mul(dag(L(nu, 0, -1)), L(mu, 0, -1)), mul(L(nu, 1, -1), dag(L(mu, 0, 0))));
  cpx<double> tr = {0, 0};
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) {
      cpx<double> qab = l1.m[a][b] + l2.m[a][b] + l3.m[a][b] + l4.m[a][b];
      cpx<double> qba = l1.m[b][a] + l2.m[b][a] + l3.m[b][a] + l4.m[b][a];
      F.m[a][b] = 0.125 * (qab - conj(qba));
    }
  for (int a = 0; a < 3; a++) tr = tr + F.m[a][a];
  for (int a = 0; a < 3; a++) F.m[a][a] = F.m[a][a] - (1.0 / 3.0) * tr;
}

__device__ bool invert6(cpx<double> a[6][6], cpx<double> inv[6][6]) {
  for (int i = 0; i < 6; i++)
    for (int j = 0; j < 6; j++) inv[i][j] = {i == j ? 1.0 : 0.0, 0.0};
  for (int col = 0; col < 6; col++) {
    int piv = col;
    double best = 0;
    for (int r = col; r < 6; r++) {
      double m = a[r][col].re * a[r][col].re + a[r][col].im * a[r][col].im;
      if (m > best) {
        best = m;
        piv = r;
      }
    }
    if (!(best > 0)) return false;
    if (piv != col)
      for (int j = 0; j < 6; j++) {
        cpx<double> t = a[col][j];
        a[col][j] = a[piv][j];
        a[piv][j] = t;
        t = inv[col][j];
        inv[col][j] = inv[piv][j];
        inv[piv][j] = t;
      }
    const cpx<double> d = a[col][col];
    const double dn = d.re * d.re + d.im * d.im;
    const cpx<double> rinv = {d.re / dn, -d.im / dn};
    for (int j = 0; j < 6; j++) {
      a[col][j] = a[col][j] * rinv;
      inv[col][j] = inv[col][j] * rinv;
    }
    for (int r = 0; r < 6; r++) {
      if (r == col) continue;
      const cpx<double> f = a[r][col];
      for (int j = 0; j < 6; j++) {
        a[r][j] = a[r][j] - f * a[col][j];
        inv[r][j] = inv[r][j] - f * inv[col][j];
      }
    }
  }
  return true;
}

__device__ void pack_block(double2* dst, long st, long i, int b, const cpx<double> m[6][6]) {
  // 3 double2 of diagonal pairs, then 15 lower entries
  for (int k = 0; k < 3; k++) dst[(18 * b + k) * st + i] = make_double2(m[2 * k][2 * k].re, m[2 * k + 1][2 * k + 1].re);
  int k = 0;
  for (int r = 1; r < 6; r++)
    for (int c = 0; c < r; c++, k++) dst[(18 * b + 3 + k) * st + i] = make_double2(m[r][c].re, m[r][c].im);
}

// csw_t multiplies the planes (mu, 3) that contain t, csw_s the spatial planes
__global__ void clover_build_kernel(const double2* __restrict__ qdp, QdpGeom q, double kappa, double csw_t,
                                    double csw_s,
                                    double2* A0, double2* A1, double2* Ai0, double2* Ai1, long st,
                                    int* __restrict__ flags) {
  const long n = 2 * q.vh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int p = (int)(idx / q.vh);
    const long i = idx % q.vh;
    int c[4];
    site_coords(q, p, i, c[0], c[1], c[2], c[3]);
    cpx<double> blk[2][6][6];
    for (int b = 0; b < 2; b++)
      for (int r = 0; r < 6; r++)
        for (int cc = 0; cc < 6; cc++) blk[b][r][cc] = {r == cc ? 1.0 : 0.0, 0.0};
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) {
        Mat3 F;
        field_strength(qdp, q, mu, nu, c, F);
        // sigma_{mu nu} = (g_mu g_nu - g_nu g_mu) / 2
        cpx<double> sg[4][4];
        for (int a = 0; a < 4; a++)
          for (int b = 0; b < 4; b++) {
            cpx<double> s = {0, 0};
            for (int k = 0; k < 4; k++) {
              cpx<double> gm_ak = {c_gamma[mu][a][k][0], c_gamma[mu][a][k][1]};
              cpx<double> gn_kb = {c_gamma[nu][k][b][0], c_gamma[nu][k][b][1]};
              cpx<double> gn_ak = {c_gamma[nu][a][k][0], c_gamma[nu][a][k][1]};
              cpx<double> gm_kb = {c_gamma[mu][k][b][0], c_gamma[mu][k][b][1]};
              s = s + gm_ak * gn_kb - gn_ak * gm_kb;
            }
            sg[a][b] = 0.5 * s;
          }
        for (int b = 0; b < 2; b++)
          for (int s1 = 0; s1 < 2; s1++)
            for (int s2 = 0; s2 < 2; s2++) {
              const cpx<double> sv = (-kappa * (nu == 3 ? csw_t : csw_s)) * sg[2 * b + s1][2 * b + s2];
              for (int ca = 0; ca < 3; ca++)
                for (int cb = 0; cb < 3; cb++) blk[b][3 * s1 + ca][3 * s2 + cb] = blk[b][3 * s1 + ca][3 * s2 + cb] + sv * F.m[ca][cb];
            }
      }
    double2* A = p ? A1 : A0;
    double2* Ai = p ? Ai1 : Ai0;
    for (int b = 0; b < 2; b++) {
      pack_block(A, st, i, b, blk[b]);
      cpx<double> inv[6][6];
      if (!invert6(blk[b], inv)) atomicOr(flags, 4);
      pack_block(Ai, st, i, b, inv);
    }
  }
}

// F64 packed clover -> F32 / F16 / BF16 copies (half: one FP32 scale per site)
__global__ void clover_pack_kernel(const double2* __restrict__ src, long st, long vh, float4* d32, uint4* d16,
                                   float* n16, uint4* db16, float* nb16) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < vh; i += (long)gridDim.x * blockDim.x) {
    double r[72];
    for (int k = 0; k < 36; k++) {
      double2 v = src[k * st + i];
      r[2 * k] = v.x;
      r[2 * k + 1] = v.y;
    }
    for (int k = 0; k < 18; k++) d32[k * st + i] = make_float4((float)r[4 * k], (float)r[4 * k + 1], (float)r[4 * k + 2], (float)r[4 * k + 3]);
    double m = 0;
    for (int k = 0; k < 72; k++) m = fmax(m, fabs(r[k]));
    const double inv = m > 0 ? 1.0 / m : 0.0;
    n16[i] = (float)m;
    nb16[i] = (float)m;
    for (int k = 0; k < 9; k++) {
      uint4 a, b;
      a.x = pack2<F16>((float)(r[8 * k + 0] * inv), (float)(r[8 * k + 1] * inv));
      a.y = pack2<F16>((float)(r[8 * k + 2] * inv), (float)(r[8 * k + 3] * inv));
      a.z = pack2<F16>((float)(r[8 * k + 4] * inv), (float)(r[8 * k + 5] * inv));
      a.w = pack2<F16>((float)(r[8 * k + 6] * inv), (float)(r[8 * k + 7] * inv));
      b.x = pack2<BF16>((float)(r[8 * k + 0] * inv), (float)(r[8 * k + 1] * inv));
      b.y = pack2<BF16>((float)(r[8 * k + 2] * inv), (float)(r[8 * k + 3] * inv));
      b.z = pack2<BF16>((float)(r[8 * k + 4] * inv), (float)(r[8 * k + 5] * inv));
      b.w = pack2<BF16>((float)(r[8 * k + 6] * inv), (float)(r[8 * k + 7] * inv));
      d16[k * st + i] = a;
      db16[k * st + i] = b;
    }
  }
}

// ---------------------------------------------------------------------------
// fermion import / export between QDP complex128 and internal F64 parity fields.
//   src element (rhs, i, k) at src + rhs*rhs_stride + par_off + i*12 + k
// QDP fermion (12 complexes per site, site-major) <-> internal chunk-major layout,
// through a shared-memory tile of 32 sites so that both the QDP side (which may be
// page-locked host memory read over the host link) and the chunk side move in
// contiguous runs: the QDP run of a tile is 32 x 12 consecutive complexes.
constexpr int FIO_SITES = 32;

__global__ void __launch_bounds__(128) fermion_import_kernel(const double2* __restrict__ src, long rhs_stride,
                                                             long par_off, long vh, int nrhs, double2* __restrict__ dst,
                                                             long st, int* __restrict__ flags) {
  __shared__ double2 tile[12][FIO_SITES + 1];
  const long ntile = (vh + FIO_SITES - 1) / FIO_SITES;
  bool fin = true;
  for (long tix = blockIdx.x; tix < (long)nrhs * ntile; tix += gridDim.x) {
    const int r = (int)(tix / ntile);
    const long i0 = (tix % ntile) * FIO_SITES;
    const int ns = (int)((vh - i0) < FIO_SITES ? (vh - i0) : FIO_SITES);
    const double2* s = src + r * rhs_stride + par_off + i0 * 12;
    for (int e = threadIdx.x; e < ns * 12; e += blockDim.x) {
      const double2 v = s[e];
      fin = fin && isfinite(v.x) && isfinite(v.y);
      tile[e % 12][e / 12] = v;
    }
    __syncthreads();
    double2* d = dst + (long)r * 12 * st + i0;
    for (int e = threadIdx.x; e < 12 * FIO_SITES; e += blockDim.x) {
      const int k = e / FIO_SITES, site = e % FIO_SITES;
      if (site < ns) d[k * st + site] = tile[k][site];
    }
    __syncthreads();
  }
  if (!fin && flags) atomicOr(flags, 1);
}

__global__ void __launch_bounds__(128) fermion_export_kernel(const double2* __restrict__ src, long st, long vh,
                                                             int nrhs, double2* __restrict__ dst, long rhs_stride,
                                                             long par_off) {
  __shared__ double2 tile[12][FIO_SITES + 1];
  const long ntile = (vh + FIO_SITES - 1) / FIO_SITES;
  for (long tix = blockIdx.x; tix < (long)nrhs * ntile; tix += gridDim.x) {
    const int r = (int)(tix / ntile);
    const long i0 = (tix % ntile) * FIO_SITES;
    const int ns = (int)((vh - i0) < FIO_SITES ? (vh - i0) : FIO_SITES);
    const double2* s = src + (long)r * 12 * st + i0;
    for (int e = threadIdx.x; e < 12 * FIO_SITES; e += blockDim.x) {
      const int k = e / FIO_SITES, site = e % FIO_SITES;
      if (site < ns) tile[k][site] = s[k * st + site];
    }
    __syncthreads();
    double2* d = dst + r * rhs_stride + par_off + i0 * 12;
    for (int e = threadIdx.x; e < ns * 12; e += blockDim.x) d[e] = tile[e % 12][e / 12];
    __syncthreads();
  }
}

// [12][site][Ns][Nc] (source k = 3 s0 + c0) <-> [site][Ns][Ns][Nc][Nc]: one thread per
// (site, 16-byte complex) of the propagator; to_prop selects the direction
__global__ void propagator_kernel(const double2* __restrict__ src, double2* __restrict__ dst, long nsite, int to_prop) {
  const long n = nsite * 144;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const long site = e / 144;
    const int q = (int)(e % 144);  // propagator index ((s * 4 + s0) * 3 + c) * 3 + c0
    const int c0 = q % 3, c = (q / 3) % 3, s0 = (q / 9) % 4, s = q / 36;
    const long f = ((long)(3 * s0 + c0) * nsite + site) * 12 + 3 * s + c;  // fermion index
    if (to_prop)
      dst[e] = src[f];
    else
      dst[f] = src[e];
  }
}

// ---------------------------------------------------------------------------
static int grid_for(long n, int block) {
  long g = (n + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  return (int)(g < 1 ? 1 : g);
}

static QdpGeom qgeom(const LatticeDevice& L) {
  QdpGeom q;
  q.Lx = L.dims[0];
  q.Ly = L.dims[1];
  q.Lz = L.dims[2];
  q.Lt = L.dims[3];
  q.lxh = L.dims[0] / 2;
  q.vh = L.vh;
  return q;
}

// double-float copy: every FP64 real d becomes (hi, lo) = (fl(d), fl(d - fl(d)))
__global__ void split_df64_kernel(const double2* __restrict__ src, float4* __restrict__ dst, long n) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const double2 d = src[k];
    const float rh = (float)d.x, ih = (float)d.y;
    dst[k] = make_float4(rh, (float)(d.x - (double)rh), ih, (float)(d.y - (double)ih));
  }
}

static cudaError_t split_df64(const void* src, void* dst, size_t bytes, cudaStream_t st) {
  const long n = (long)(bytes / 16);
  split_df64_kernel<<<grid_for(n, 256), 256, 0, st>>>(static_cast<const double2*>(src), static_cast<float4*>(dst), n);
  return cudaGetLastError();
}

cudaError_t import_gauge(const LatticeDevice& L, const void* d_qdp, int* d_flags, cudaStream_t st) {
  GaugePack gp;
  for (int p = 0; p < 2; p++) {
    gp.g64[p] = L.gauge[F64][p];
    gp.g32[p] = L.gauge[F32][p];
    gp.g16[p] = L.gauge[F16][p];
    gp.gb16[p] = L.gauge[BF16][p];
  }
  gp.stride = L.stride;
  gauge_import_kernel<<<grid_for(8 * L.vh, 256), 256, 0, st>>>(static_cast<const double2*>(d_qdp), qgeom(L), gp, 1e-12,
                                                               d_flags);
  cudaError_t e = cudaGetLastError();
  for (int p = 0; p < 2 && e == cudaSuccess; p++)
    e = split_df64(L.gauge[F64][p], L.gauge[DF64][p], gauge_parity_bytes(F64, L.stride), st);
  return e;
}

cudaError_t build_clover(const LatticeDevice& L, const void* d_qdp, double kappa, double csw_t, double csw_s,
                         int* d_flags, cudaStream_t st) {
  clover_build_kernel<<<grid_for(2 * L.vh, 64), 64, 0, st>>>(
      static_cast<const double2*>(d_qdp), qgeom(L), kappa, csw_t, csw_s, static_cast<double2*>(L.clov[F64][0]),
      static_cast<double2*>(L.clov[F64][1]), static_cast<double2*>(L.clovinv[F64][0]),
      static_cast<double2*>(L.clovinv[F64][1]), L.stride, d_flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int p = 0; p < 2; p++) {
    for (int inv = 0; inv < 2; inv++) {
      float* const* nrm = inv ? L.clovinv_norm : L.clov_norm;
      const double2* src = static_cast<const double2*>(inv ? L.clovinv[F64][p] : L.clov[F64][p]);
      clover_pack_kernel<<<grid_for(L.vh, 128), 128, 0, st>>>(
          src, L.stride, L.vh, static_cast<float4*>(inv ? L.clovinv[F32][p] : L.clov[F32][p]),
          static_cast<uint4*>(inv ? L.clovinv[F16][p] : L.clov[F16][p]), nrm[F16 * 2 + p],
          static_cast<uint4*>(inv ? L.clovinv[BF16][p] : L.clov[BF16][p]), nrm[BF16 * 2 + p]);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      e = split_df64(src, inv ? L.clovinv[DF64][p] : L.clov[DF64][p], clover_parity_bytes(F64, L.stride), st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t import_fermion(const LatticeDevice& L, const void* d_src, long rhs_stride_c, long par_off_c, int nrhs,
                           void* d_dst64, int* d_flags, cudaStream_t st) {
  fermion_import_kernel<<<grid_for((long)nrhs * ((L.vh + FIO_SITES - 1) / FIO_SITES), 1), 128, 0, st>>>(
      static_cast<const double2*>(d_src), rhs_stride_c, par_off_c, L.vh, nrhs, static_cast<double2*>(d_dst64), L.stride,
      d_flags);
  return cudaGetLastError();
}

cudaError_t export_fermion(const LatticeDevice& L, const void* d_src64, int nrhs, void* d_dst, long rhs_stride_c,
                           long par_off_c, cudaStream_t st) {
  fermion_export_kernel<<<grid_for((long)nrhs * ((L.vh + FIO_SITES - 1) / FIO_SITES), 1), 128, 0, st>>>(
      static_cast<const double2*>(d_src64), L.stride, L.vh, nrhs, static_cast<double2*>(d_dst), rhs_stride_c, par_off_c);
  return cudaGetLastError();
}

}  // namespace wcl

namespace wcl {
cudaError_t propagator_layout(const LatticeDevice& L, const void* src, void* dst, int to_prop, cudaStream_t st) {
  const long nsite = 2 * L.vh;
  propagator_kernel<<<grid_for(nsite * 144, 256), 256, 0, st>>>(static_cast<const double2*>(src),
                                                                static_cast<double2*>(dst), nsite, to_prop);
  return cudaGetLastError();
}
}  // namespace wcl
