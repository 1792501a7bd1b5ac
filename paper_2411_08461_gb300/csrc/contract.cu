// Propagator workflow around the solve (Sec. III.A, III.B): wall and momentum
// sources, the sequential source (Eq. 4 and the sequential-source equation of
// Sec. III.B) and the meson contractions of Eq. 6 and Eq. 7, on QDP-layout
// complex128 fields:
//   fermion    [2][Lt][Lz][Ly][Lx/2][4][3]
//   propagator [2][Lt][Lz][Ly][Lx/2][4][4][3][3]  (sink spin, source spin, sink colour, source colour)
//
// Momentum: p_k = 2 pi n_k / L_k.  The momentum wall source carries exp(+i p.x) and
// the sink of a contraction and the sequential source exp(-i p.x) (the source and
// sink phases of Eq. 1 and Eq. 2).
//
// Gamma matrices: the calls take a 4x4 complex matrix with exactly one nonzero entry
// per row, equal to 1, i, -1 or -i -- every product of DeGrand-Rossi gamma matrices
// has this form -- stored as a column index and a power of i per row.
//
// The contraction of two complex128 propagators moves 4608 bytes per site and does
// 576 double-precision FMAs; on a GPU whose FP64 rate is about 2 FMAs per clock per
// SM that is the binding resource, so the kernel spends as little FP64 work as
// possible beyond those FMAs: the Gamma entries are applied as sign and swap, the
// phase once per (site, lane).
#include <cmath>
#include <cstring>

#include "context.cuh"

wcl_status wcl_enter(wcl_ctx* c);
wcl_status wcl_leave(wcl_ctx* c, wcl_status s);
bool wcl_resolve_field(const wcl_ctx* c, const void* p, const void** out, const char* what);

namespace wcl {
namespace {

struct SiteGeom {
  int Lx, Ly, Lz, Lt;
  int vs2;  // sites per parity per timeslice, Lz * Ly * Lx / 2
  long vh;  // sites per parity
};

struct Mom {
  int n[3];
};

// Gamma row i: Gamma[i][col[i]] = i^rot[i], every other entry zero
struct GammaRows {
  int col[4];
  int rot[4];
};

SiteGeom geom_of(const LatticeDevice& L) {
  SiteGeom g;
  g.Lx = L.dims[0], g.Ly = L.dims[1], g.Lz = L.dims[2], g.Lt = L.dims[3];
  g.vs2 = L.dims[2] * L.dims[1] * (L.dims[0] / 2);
  g.vh = L.vh;
  return g;
}

// storage site (parity-major) -> lattice coordinates
__device__ __forceinline__ void site_coords(const SiteGeom& g, long site, int& x, int& y, int& z, int& t) {
  const int par = site >= g.vh;
  int cb = (int)(site - (par ? g.vh : 0));
  const int hx = g.Lx / 2;
  const int xh = cb % hx;
  cb /= hx;
  y = cb % g.Ly;
  cb /= g.Ly;
  z = cb % g.Lz;
  t = cb / g.Lz;
  x = 2 * xh + ((y + z + t + par) & 1);
}

__device__ __forceinline__ long long mod_pos(long long a, long long L) {
  const long long r = a % L;
  return r < 0 ? r + L : r;
}

// exp(sign * i p.x): the argument p.x / 2 pi is reduced exactly in integers, then
// rounded once by the division before sincospi
__device__ __forceinline__ double2 plane_wave(const SiteGeom& g, const Mom& m, int sign, int x, int y, int z) {
  const long long lx = g.Lx, ly = g.Ly, lz = g.Lz, den = lx * ly * lz;
  long long num = mod_pos((long long)m.n[0] * x, lx) * ly * lz + mod_pos((long long)m.n[1] * y, ly) * lx * lz +
                  mod_pos((long long)m.n[2] * z, lz) * lx * ly;
  num %= den;
  double s, c;
  sincospi(2.0 * (double)num / (double)den, &s, &c);
  return make_double2(c, sign > 0 ? s : -s);
}

// v * i^r
__device__ __forceinline__ double2 rot_i(double2 v, int r) {
  const bool sw = r & 1;
  const double a = sw ? v.y : v.x, b = sw ? v.x : v.y;
  return make_double2((r == 1 || r == 2) ? -a : a, r >= 2 ? -b : b);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// twelve wall sources: fermion k = 3 s + c holds the phase (or 1) in spin s, colour c
// on timeslice t0; one thread per complex element, blockIdx.y = k
__global__ void wall_source_kernel(double2* __restrict__ b, SiteGeom g, Mom m, int t0, int with_phase) {
  const int k = blockIdx.y;
  const long nel = 2 * g.vh * 12;
  double2* out = b + (long)k * nel;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nel; e += (long)gridDim.x * blockDim.x) {
    const long site = e / 12;
    const int q = (int)(e - site * 12);
    double2 v = make_double2(0.0, 0.0);
    if (q == k) {
      int x, y, z, t;
      site_coords(g, site, x, y, z, t);
      if (t == t0) v = with_phase ? plane_wave(g, m, +1, x, y, z) : make_double2(1.0, 0.0);
    }
    __stcs(out + e, v);
  }
}

// X[i][k][a][b] = exp(-i p.x) Gamma[i][j] S[j][k][a][b] on timeslice ts, zero elsewhere
__global__ void sequential_source_kernel(double2* __restrict__ X, const double2* __restrict__ S, SiteGeom g, Mom m,
                                         int ts, int with_phase, GammaRows gr) {
  const long nel = 2 * g.vh * 144;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nel; e += (long)gridDim.x * blockDim.x) {
    const long site = e / 144;
    const int q = (int)(e - site * 144);
    int x, y, z, t;
    site_coords(g, site, x, y, z, t);
    double2 v = make_double2(0.0, 0.0);
    if (t == ts) {
      const int i = q / 36, r = q - i * 36;
      v = rot_i(__ldcs(S + site * 144 + gr.col[i] * 36 + r), gr.rot[i]);
      if (with_phase) v = cmul(v, plane_wave(g, m, -1, x, y, z));
    }
    __stcs(X + e, v);
  }
}

// exp(-i p.x) at every storage site
__global__ void phase_table_kernel(double2* __restrict__ ph, SiteGeom g, Mom m) {
  const long n = 2 * g.vh;
  for (long s = blockIdx.x * (long)blockDim.x + threadIdx.x; s < n; s += (long)gridDim.x * blockDim.x) {
    int x, y, z, t;
    site_coords(g, s, x, y, z, t);
    ph[s] = plane_wave(g, m, -1, x, y, z);
  }
}

// ---- contraction ------------------------------------------------------------------
// A run is the contiguous storage range of one (parity, timeslice).  A CTA takes
// `tiles_per_block` consecutive tiles of CT_SITES sites from one run; each of its
// CT_WARPS warps owns one shared-memory stage and loads its tiles into it with
// cp.async (16-byte copies, coalesced), single-buffered: the warps of the SM (twelve
// at 37 KB per CTA) hide each other's loads.  Lane (h, s, i) then reads rows 2h and
// 2h+1 of site s, source spin i: nine colour pairs each of A and of the B row that
// Gamma selects (padded site rows keep the 16-byte shared-memory reads conflict-free).
// Each CTA writes one partial sum; the finaliser adds them per timeslice in a fixed
// order (deterministic).
constexpr int CT_SITES = 4;
constexpr int CT_ROW = 148;                          // double2 per staged site: 144 + 4 padding
constexpr int CT_STAGE = 2 * CT_SITES * CT_ROW;      // A and B of one tile
constexpr int CT_WARPS = 2;
constexpr size_t CT_SMEM = CT_WARPS * CT_STAGE * sizeof(double2);

struct ContractArgs {
  const double2* A;
  const double2* B;
  const double2* ph;  // exp(-i p.x) per storage site, nullptr for p = 0
  double2* partials;  // [run][chunk]
  GammaRows gr;
  long vh;
  int vs2, lt;
  int tiles_per_run, tiles_per_block, chunks;
};

__device__ __forceinline__ void contract_issue(const ContractArgs& a, double2* dst, long run_base, int first,
                                               int lane) {
  const int ns = min(CT_SITES, a.vs2 - first);
#pragma unroll 4
  for (int e = lane; e < 2 * CT_SITES * 144; e += 32) {
    const int p = e / (CT_SITES * 144);
    const int rem = e - p * (CT_SITES * 144);
    const int ss = rem / 144, q = rem - ss * 144;
    if (ss < ns) cp_async16(dst + (p * CT_SITES + ss) * CT_ROW + q, (p ? a.B : a.A) + (run_base + first + ss) * 144 + q);
  }
  cp_async_commit();
}

__global__ void __launch_bounds__(32 * CT_WARPS) contract_kernel(ContractArgs a) {
  extern __shared__ double2 ct_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double2* stage = ct_smem + warp * CT_STAGE;
  const int run = blockIdx.y;
  const int par = run / a.lt, t = run - par * a.lt;
  const long run_base = (long)par * a.vh + (long)t * a.vs2;
  const int tile0 = blockIdx.x * a.tiles_per_block;
  const int ntile = min(a.tiles_per_block, a.tiles_per_run - tile0);
  const int h = lane >> 4, s = (lane >> 2) & 3, i = lane & 3;
  const int j0 = 2 * h, j1 = 2 * h + 1;
  // constant indices keep the Gamma rows in registers
  const int c0 = h ? a.gr.col[2] : a.gr.col[0], c1 = h ? a.gr.col[3] : a.gr.col[1];
  const int r0 = h ? a.gr.rot[2] : a.gr.rot[0], r1 = h ? a.gr.rot[3] : a.gr.rot[1];

  double tr = 0.0, ti = 0.0;
  for (int tl = warp; tl < ntile; tl += CT_WARPS) {
    const int first = (tile0 + tl) * CT_SITES;
    contract_issue(a, stage, run_base, first, lane);
    cp_async_wait<0>();
    __syncwarp();
    if (first + s < a.vs2) {
      const double2* sa = stage + s * CT_ROW + i * 9;
      const double2* sb = sa + CT_SITES * CT_ROW;
      double xr0 = 0.0, xi0 = 0.0, xr1 = 0.0, xi1 = 0.0;
#pragma unroll
      for (int m = 0; m < 9; m++) {
        const double2 a0 = sa[j0 * 36 + m], b0 = sb[c0 * 36 + m];
        const double2 a1 = sa[j1 * 36 + m], b1 = sb[c1 * 36 + m];
        xr0 = fma(a0.x, b0.x, xr0);
        xr0 = fma(a0.y, b0.y, xr0);
        xi0 = fma(a0.x, b0.y, xi0);
        xi0 = fma(-a0.y, b0.x, xi0);
        xr1 = fma(a1.x, b1.x, xr1);
        xr1 = fma(a1.y, b1.y, xr1);
        xi1 = fma(a1.x, b1.y, xi1);
        xi1 = fma(-a1.y, b1.x, xi1);
      }
      const double2 u0 = rot_i(make_double2(xr0, xi0), r0), u1 = rot_i(make_double2(xr1, xi1), r1);
      const double ur = u0.x + u1.x, ui = u0.y + u1.y;
      if (a.ph) {
        const double2 p = a.ph[run_base + first + s];
        tr = fma(p.x, ur, fma(-p.y, ui, tr));
        ti = fma(p.x, ui, fma(p.y, ur, ti));
      } else {
        tr += ur;
        ti += ui;
      }
    }
    __syncwarp();  // every lane is done with the stage before it is refilled
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr += __shfl_xor_sync(0xffffffffu, tr, o);
    ti += __shfl_xor_sync(0xffffffffu, ti, o);
  }
  // each warp leaves its sum in the first slot of its own (now idle) stage: no static
  // shared memory, so six CTAs still fit on an SM
  if (lane == 0) stage[0] = make_double2(tr, ti);
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 v = ct_smem[0];
    for (int w = 1; w < CT_WARPS; w++) v.x += ct_smem[w * CT_STAGE].x, v.y += ct_smem[w * CT_STAGE].y;
    a.partials[(long)run * a.chunks + blockIdx.x] = v;
  }
}

// out[t] = sum over both parities and every chunk of the partials of timeslice t
__global__ void contract_finalize_kernel(double2* __restrict__ out, const double2* __restrict__ partials, int lt,
                                         int chunks) {
  __shared__ double sr[256], si[256];
  const int t = blockIdx.x;
  double r = 0.0, im = 0.0;
  for (int k = threadIdx.x; k < 2 * chunks; k += blockDim.x) {
    const int par = k / chunks, c = k - par * chunks;
    const double2 v = partials[(long)(par * lt + t) * chunks + c];
    r += v.x;
    im += v.y;
  }
  sr[threadIdx.x] = r;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sr[threadIdx.x] += sr[threadIdx.x + w];
      si[threadIdx.x] += si[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[t] = make_double2(sr[0], si[0]);
}

int grid_1d(long n, int block) {
  long g = (n + block - 1) / block;
  if (g > 152 * 16) g = 152 * 16;
  return (int)(g < 1 ? 1 : g);
}

// The DeGrand-Rossi gamma matrices gamma_1 .. gamma_4 (Chroma convention), row-major,
// entries (re, im).
const double kGammaDR[4][16][2] = {
    {{0, 0}, {0, 0}, {0, 0}, {0, 1}, {0, 0}, {0, 0}, {0, 1}, {0, 0},
     {0, 0}, {0, -1}, {0, 0}, {0, 0}, {0, -1}, {0, 0}, {0, 0}, {0, 0}},
    {{0, 0}, {0, 0}, {0, 0}, {-1, 0}, {0, 0}, {0, 0}, {1, 0}, {0, 0},
     {0, 0}, {1, 0}, {0, 0}, {0, 0}, {-1, 0}, {0, 0}, {0, 0}, {0, 0}},
    {{0, 0}, {0, 0}, {0, 1}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, -1},
     {0, -1}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 1}, {0, 0}, {0, 0}},
    {{0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0},
     {1, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {1, 0}, {0, 0}, {0, 0}},
};

bool parse_gamma(const double* g, GammaRows* out, const char* what) {
  for (int i = 0; i < 4; i++) {
    int found = -1;
    for (int j = 0; j < 4; j++) {
      const double re = g[2 * (4 * i + j)], im = g[2 * (4 * i + j) + 1];
      if (!std::isfinite(re) || !std::isfinite(im)) {
        set_error("%s: non-finite Gamma entry", what);
        return false;
      }
      if (std::fabs(re) <= 1e-12 && std::fabs(im) <= 1e-12) continue;
      int r = -1;
      if (std::fabs(re - 1) <= 1e-12 && std::fabs(im) <= 1e-12) r = 0;
      if (std::fabs(re) <= 1e-12 && std::fabs(im - 1) <= 1e-12) r = 1;
      if (std::fabs(re + 1) <= 1e-12 && std::fabs(im) <= 1e-12) r = 2;
      if (std::fabs(re) <= 1e-12 && std::fabs(im + 1) <= 1e-12) r = 3;
      if (r < 0 || found >= 0) {
        set_error("%s: Gamma must have one entry 1, i, -1 or -i per row and zeros elsewhere", what);
        return false;
      }
      found = j;
      out->col[i] = j;
      out->rot[i] = r;
    }
    if (found < 0) {
      set_error("%s: Gamma row %d is zero", what, i);
      return false;
    }
  }
  return true;
}

// propagators read by cp.async must be device memory of the context's GPU
bool device_field(const wcl_ctx* c, const void* p, const char* what) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    set_error("%s: not a CUDA-accessible pointer", what);
    return false;
  }
  if ((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == c->device) return true;
  set_error("%s: the propagators must be device memory of the context's GPU", what);
  return false;
}

bool parse_mom(const int* mom, Mom* m) {
  for (int k = 0; k < 3; k++) m->n[k] = mom ? mom[k] : 0;
  return mom && (m->n[0] || m->n[1] || m->n[2]);
}

}  // namespace
}  // namespace wcl

using namespace wcl;

extern "C" {

wcl_status wcl_gamma(int n, double* h_out) {
  if (n < 0 || n > 15 || !h_out) {
    set_error("wcl_gamma: n must be 0..15 and h_out non-null");
    return WCL_ERR_INVALID_ARG;
  }
  double m[4][4][2] = {};
  for (int i = 0; i < 4; i++) m[i][i][0] = 1.0;
  for (int k = 0; k < 4; k++) {
    if (!((n >> k) & 1)) continue;
    double r[4][4][2] = {};
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++)
        for (int l = 0; l < 4; l++) {
          const double ar = m[i][l][0], ai = m[i][l][1];
          const double br = kGammaDR[k][4 * l + j][0], bi = kGammaDR[k][4 * l + j][1];
          r[i][j][0] += ar * br - ai * bi;
          r[i][j][1] += ar * bi + ai * br;
        }
    std::memcpy(m, r, sizeof(m));
  }
  std::memcpy(h_out, m, sizeof(m));
  return WCL_OK;
}

wcl_status wcl_kappa_from_mass(double m0, double* kappa) {
  if (!kappa || !std::isfinite(m0) || !(m0 + 4.0 > 0.0)) {
    set_error("wcl_kappa_from_mass: need a finite m0 > -4 and a non-null output");
    return WCL_ERR_INVALID_ARG;
  }
  *kappa = 1.0 / (2.0 * (m0 + 4.0));
  return WCL_OK;
}

wcl_status wcl_kappa_from_mass_aniso(double m0, double xi0, double nu, double* kappa) {
  const double d = m0 + 1.0 + 3.0 * nu / xi0;
  if (!kappa || !std::isfinite(m0) || !std::isfinite(xi0) || !std::isfinite(nu) || !(xi0 > 0) || !(nu > 0) ||
      !(d > 0)) {
    set_error("wcl_kappa_from_mass_aniso: need finite m0, positive xi0 and nu, and m0 + 1 + 3 nu/xi0 > 0");
    return WCL_ERR_INVALID_ARG;
  }
  *kappa = 1.0 / (2.0 * d);
  return WCL_OK;
}

wcl_status wcl_wall_source(wcl_ctx* c, void* d_b12, int t0, const int* mom) {
  if (!c || !d_b12 || t0 < 0 || t0 >= c->lat.dims[3]) {
    set_error("wcl_wall_source: invalid argument (t0 must be 0..Lt-1)");
    return WCL_ERR_INVALID_ARG;
  }
  const void* p = nullptr;
  if (!wcl_resolve_field(c, d_b12, &p, "wcl_wall_source")) return WCL_ERR_INVALID_ARG;
  Mom m;
  const bool with_phase = parse_mom(mom, &m);
  WCL_CHECK(wcl_enter(c));
  const SiteGeom g = geom_of(c->lat);
  wall_source_kernel<<<dim3(grid_1d(2 * g.vh * 12, 256), 12), 256, 0, c->stream>>>(
      static_cast<double2*>(const_cast<void*>(p)), g, m, t0, with_phase);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  return wcl_leave(c, WCL_OK);
}

wcl_status wcl_sequential_source(wcl_ctx* c, void* d_X, const void* d_S, int t, const int* mom,
                                 const double* h_gamma) {
  if (!c || !d_X || !d_S || d_X == d_S || t < 0 || t >= c->lat.dims[3]) {
    set_error("wcl_sequential_source: invalid argument (distinct buffers, t must be 0..Lt-1)");
    return WCL_ERR_INVALID_ARG;
  }
  GammaRows gr;
  if (h_gamma) {
    if (!parse_gamma(h_gamma, &gr, "wcl_sequential_source")) return WCL_ERR_INVALID_ARG;
  } else {
    double g5[32];
    wcl_gamma(15, g5);
    parse_gamma(g5, &gr, "wcl_sequential_source");
  }
  const void *px = nullptr, *ps = nullptr;
  if (!wcl_resolve_field(c, d_X, &px, "wcl_sequential_source") || !wcl_resolve_field(c, d_S, &ps, "wcl_sequential_source"))
    return WCL_ERR_INVALID_ARG;
  Mom m;
  const bool with_phase = parse_mom(mom, &m);
  WCL_CHECK(wcl_enter(c));
  const SiteGeom g = geom_of(c->lat);
  sequential_source_kernel<<<grid_1d(2 * g.vh * 144, 256), 256, 0, c->stream>>>(
      static_cast<double2*>(const_cast<void*>(px)), static_cast<const double2*>(ps), g, m, t, with_phase, gr);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  return wcl_leave(c, WCL_OK);
}

wcl_status wcl_contract(wcl_ctx* c, void* d_out, const void* d_A, const void* d_B, const double* h_gamma,
                        const int* mom) {
  if (!c || !d_out || !d_A || !d_B) {
    set_error("wcl_contract: invalid argument");
    return WCL_ERR_INVALID_ARG;
  }
  GammaRows gr;
  if (h_gamma) {
    if (!parse_gamma(h_gamma, &gr, "wcl_contract")) return WCL_ERR_INVALID_ARG;
  } else {
    for (int i = 0; i < 4; i++) gr.col[i] = i, gr.rot[i] = 0;
  }
  const void *po = nullptr, *pa = nullptr, *pb = nullptr;
  if (!wcl_resolve_field(c, d_out, &po, "wcl_contract") || !device_field(c, d_A, "wcl_contract") ||
      !device_field(c, d_B, "wcl_contract"))
    return WCL_ERR_INVALID_ARG;
  pa = d_A, pb = d_B;
  Mom m;
  const bool with_phase = parse_mom(mom, &m);
  const SiteGeom g = geom_of(c->lat);
  ContractArgs a;
  a.A = static_cast<const double2*>(pa);
  a.B = static_cast<const double2*>(pb);
  a.gr = gr;
  a.vh = g.vh;
  a.vs2 = g.vs2;
  a.lt = g.Lt;
  a.tiles_per_run = (g.vs2 + CT_SITES - 1) / CT_SITES;
  const long total_tiles = 2L * g.Lt * a.tiles_per_run;
  long tpb = (total_tiles + 152 * 5 * 4 - 1) / (152 * 5 * 4);
  a.tiles_per_block = (int)(tpb < 1 ? 1 : (tpb > 64 ? 64 : tpb));
  a.chunks = (a.tiles_per_run + a.tiles_per_block - 1) / a.tiles_per_block;
  WCL_CHECK(wcl_enter(c));
  void* part = nullptr;
  WCL_CHECK(ws_get(c, "ct_partials", sizeof(double2) * 2 * g.Lt * (size_t)a.chunks, &part));
  a.partials = static_cast<double2*>(part);
  a.ph = nullptr;
  if (with_phase) {
    void* ph = nullptr;
    WCL_CHECK(ws_get(c, "ct_phase", sizeof(double2) * 2 * (size_t)g.vh, &ph));
    phase_table_kernel<<<grid_1d(2 * g.vh, 256), 256, 0, c->stream>>>(static_cast<double2*>(ph), g, m);
    WCL_CUDA(cudaGetLastError());
    count_launch(c);
    a.ph = static_cast<const double2*>(ph);
  }
  // the CTAs are bounded by shared memory: ask for the largest carveout so that six
  // fit on an SM
  WCL_CUDA(cudaFuncSetAttribute(contract_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared));
  contract_kernel<<<dim3(a.chunks, 2 * g.Lt), 32 * CT_WARPS, CT_SMEM, c->stream>>>(a);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  contract_finalize_kernel<<<g.Lt, 256, 0, c->stream>>>(static_cast<double2*>(const_cast<void*>(po)), a.partials,
                                                        g.Lt, a.chunks);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  return wcl_leave(c, WCL_OK);
}

}  // extern "C"
