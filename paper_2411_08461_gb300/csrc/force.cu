// Fermion force of the two-flavour even-odd clover action (the HMC force of Sec. IV),
// in FP64:
//
//   S(U) = phi^+ (M_hat^+ M_hat)^-1 phi  -  2 sum_{x odd} log det A(x)      (det term optional)
//
// For U_mu(x) -> exp(eps Q) U_mu(x), Q traceless anti-Hermitian, dS/d eps = -Tr(Q F_mu(x)):
// F_mu(x) = -TA(U_mu(x) G_mu(x)) with dS = Re sum Tr(dU G).  Given X = (M_hat^+ M_hat)^-1 phi
// (even sites), with Y = M_hat X, Z = A_oo^-1 D_oe X and W = A_oo^-1 (D^+ Y)_odd:
//
//   hopping:  G += 2 kappa^2 eta { Tr_s[(1 - g_mu) B(x+mu) A(x)^+] + Tr_s[(1 + g_mu) B(x) A(x+mu)^+]^+ }
//             with A = Y (even) + W (odd), B = X (even) + Z (odd);
//   clover:   dA = -kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) dF_{mu nu}; the spin-traced
//             Xi_{mu nu}(x) = Tr_s[sigma_{mu nu} X Y^+] (even x), kappa^2 Tr_s[sigma Z W^+]
//             + Tr_s[sigma A^-1] (odd x) gives Omega = (2 kappa c_sw / 8)(Xi0 - Xi0^+)
//             (Xi0 its traceless part), and every link of every clover leaf Q_{mu nu}(s)
//             receives, by the product rule, (links after it) Omega(s) (links before it),
//             daggered where the leaf holds the link as U^+.
//
// Two kernels: one thread per site builds the six Omega matrices; one thread per link
// sums the hopping term and the 24 leaf terms (3 planes x 4 leaves x 2 positions) and
// projects.  Links are read from the context's FP64 copy, the clover inverse from its
// packed FP64 blocks.  Not on the propagator-solve path: it serves an HMC built on the
// library, so it is written for clarity at FP64, not tuned.
#include <cstring>

#include "context.cuh"

wcl_status wcl_enter(wcl_ctx* c);
wcl_status wcl_leave(wcl_ctx* c, wcl_status s);
bool wcl_resolve_field(const wcl_ctx* c, const void* p, const void** out, const char* what);

namespace wcl {
namespace {

using cd = cpx<double>;

struct M3 {
  cd m[3][3];
};

__device__ __forceinline__ M3 m3_mul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cd s = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; k++) cfma(s, a.m[i][k], b.m[k][j]);
      c.m[i][j] = s;
    }
  return c;
}
__device__ __forceinline__ M3 m3_dag(const M3& a) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) c.m[i][j] = conj(a.m[j][i]);
  return c;
}
__device__ __forceinline__ M3 m3_eye() {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) c.m[i][j] = {i == j ? 1.0 : 0.0, 0.0};
  return c;
}

// Dirac matrices (DeGrand-Rossi) and sigma_{mu nu} = [g_mu, g_nu]/2 for the six planes
// (0,1) (0,2) (0,3) (1,2) (1,3) (2,3), filled on the host
struct Spin {
  double2 gam[4][4][4];
  double2 sig[6][4][4];
};

struct ForceArgs {
  int dims[4];
  int lxh;
  long vh, stride;
  int tb;
  double kappa, csw;
  int logdet;
  const double2* gauge[2];  // FP64 links per parity: [mu][9][stride]
  const double2* ainv_odd;  // packed FP64 A^-1 of the odd sites: [36][stride]
  const double2* X;         // even   [12][stride]
  const double2* Y;         // even
  const double2* Z;         // odd
  const double2* W;         // odd
  double2* omega;           // [6 planes][9][2 vh] (parity-major sites)
  double2* out;             // QDP gauge layout [4][2][vh][9]
};

__device__ __forceinline__ void coords_of(const ForceArgs& a, int p, long i, int c[4]) {
  const int xh = (int)(i % a.lxh);
  long rem = i / a.lxh;
  c[1] = (int)(rem % a.dims[1]);
  rem /= a.dims[1];
  c[2] = (int)(rem % a.dims[2]);
  c[3] = (int)(rem / a.dims[2]);
  c[0] = 2 * xh + ((p + c[1] + c[2] + c[3]) & 1);
}

// parity and index of the site at coordinates c (wrapped periodically)
__device__ __forceinline__ void site_of(const ForceArgs& a, const int c_in[4], int& p, long& i) {
  int c[4];
#pragma unroll
  for (int d = 0; d < 4; d++) c[d] = ((c_in[d] % a.dims[d]) + a.dims[d]) % a.dims[d];
  p = (c[0] + c[1] + c[2] + c[3]) & 1;
  i = (((long)c[3] * a.dims[2] + c[2]) * a.dims[1] + c[1]) * a.lxh + (c[0] >> 1);
}

__device__ __forceinline__ M3 load_link(const ForceArgs& a, int mu, const int c[4]) {
  int p;
  long i;
  site_of(a, c, p, i);
  const double2* q = a.gauge[p] + (long)mu * 9 * a.stride + i;
  M3 u;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    const double2 v = q[k * a.stride];
    u.m[k / 3][k % 3] = {v.x, v.y};
  }
  return u;
}

__device__ __forceinline__ void load_spinor(const double2* f, long stride, long i, cd v[12]) {
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const double2 d = f[k * stride + i];
    v[k] = {d.x, d.y};
  }
}

__device__ __forceinline__ cd g2c(double2 v) { return {v.x, v.y}; }

// C_{cd} = sum_{alpha beta} g_{alpha beta} b_{beta c} conj(a_{alpha d})
__device__ __forceinline__ M3 spin_outer(const double2 g[4][4], const cd b[12], const cd a[12]) {
  M3 r;
#pragma unroll
  for (int c = 0; c < 3; c++)
#pragma unroll
    for (int d = 0; d < 3; d++) r.m[c][d] = {0.0, 0.0};
#pragma unroll
  for (int al = 0; al < 4; al++)
#pragma unroll
    for (int be = 0; be < 4; be++) {
      const cd gv = g2c(g[al][be]);
      if (gv.re == 0.0 && gv.im == 0.0) continue;
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const cd gb = gv * b[3 * be + c];
#pragma unroll
        for (int d = 0; d < 3; d++) {
          // gb * conj(a)
          const cd av = a[3 * al + d];
          r.m[c][d].re = fma(gb.re, av.re, fma(gb.im, av.im, r.m[c][d].re));
          r.m[c][d].im = fma(gb.im, av.re, fma(-gb.re, av.im, r.m[c][d].im));
        }
      }
    }
  return r;
}

// one thread per site (both parities): the six Omega_{mu nu}(x)
__global__ void __launch_bounds__(128) force_omega_kernel(const __grid_constant__ ForceArgs a,
                                                          const __grid_constant__ Spin sp) {
  const long n = 2 * a.vh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int p = (int)(idx / a.vh);
    const long i = idx % a.vh;
    cd va[12], vb[12];
    load_spinor(p == 0 ? a.Y : a.W, a.stride, i, va);
    load_spinor(p == 0 ? a.X : a.Z, a.stride, i, vb);
    const double wgt = p == 0 ? 1.0 : a.kappa * a.kappa;
    // odd sites with the determinant term: the two 6x6 blocks of A^-1 (spins 2b, 2b + 1)
    cd blk[2][6][6];
    const bool det = p == 1 && a.logdet;
    if (det) {
#pragma unroll
      for (int b = 0; b < 2; b++) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
          const double2 dg = a.ainv_odd[(18 * b + k) * a.stride + i];
          blk[b][2 * k][2 * k] = {dg.x, 0.0};
          blk[b][2 * k + 1][2 * k + 1] = {dg.y, 0.0};
        }
        int k = 0;
#pragma unroll
        for (int r = 1; r < 6; r++)
#pragma unroll
          for (int c = 0; c < r; c++, k++) {
            const cd v = g2c(a.ainv_odd[(18 * b + 3 + k) * a.stride + i]);
            blk[b][r][c] = v;
            blk[b][c][r] = conj(v);
          }
      }
    }
    const double cf = 2.0 * a.kappa * a.csw / 8.0;
    for (int pl = 0; pl < 6; pl++) {
      M3 xi = spin_outer(sp.sig[pl], vb, va);
#pragma unroll
      for (int c = 0; c < 3; c++)
#pragma unroll
        for (int d = 0; d < 3; d++) xi.m[c][d] = wgt * xi.m[c][d];
      if (det) {
        // Lambda_{cd} = sum_{alpha beta} sigma_{alpha beta} (A^-1)_{(beta c),(alpha d)}; sigma
        // commutes with gamma_5, so alpha and beta lie in the same chiral block
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
          for (int s1 = 0; s1 < 2; s1++)
#pragma unroll
            for (int s2 = 0; s2 < 2; s2++) {
              const cd sv = g2c(sp.sig[pl][2 * b + s1][2 * b + s2]);
#pragma unroll
              for (int c = 0; c < 3; c++)
#pragma unroll
                for (int d = 0; d < 3; d++) cfma(xi.m[c][d], sv, blk[b][3 * s2 + c][3 * s1 + d]);
            }
      }
      cd tr = {0.0, 0.0};
#pragma unroll
      for (int c = 0; c < 3; c++) tr = tr + xi.m[c][c];
#pragma unroll
      for (int c = 0; c < 3; c++) xi.m[c][c] = xi.m[c][c] - (1.0 / 3.0) * tr;
      double2* o = a.omega + (long)pl * 9 * n + idx;
#pragma unroll
      for (int c = 0; c < 3; c++)
#pragma unroll
        for (int d = 0; d < 3; d++) {
          const cd v = cf * (xi.m[c][d] - conj(xi.m[d][c]));
          o[(3 * c + d) * n] = make_double2(v.re, v.im);
        }
    }
  }
}

__device__ __forceinline__ M3 load_omega(const ForceArgs& a, int pl, const int c[4]) {
  int p;
  long i;
  site_of(a, c, p, i);
  const long n = 2 * a.vh;
  const double2* o = a.omega + (long)pl * 9 * n + (long)p * a.vh + i;
  M3 r;
#pragma unroll
  for (int k = 0; k < 9; k++) r.m[k / 3][k % 3] = g2c(o[k * n]);
  return r;
}

// The four leaves of Q_{mu nu}(s) with orientation +mu, +nu, -mu, -nu (Eq. 5's clover
// term): per factor, 0 = mu / 1 = nu, whether the leaf holds the link daggered, and the
// link's site relative to s in units of mu-hat and nu-hat.
struct LeafFactor {
  signed char dir, dag, om, on;
};
__constant__ LeafFactor c_leaves[4][4] = {
    {{0, 0, 0, 0}, {1, 0, 1, 0}, {0, 1, 0, 1}, {1, 1, 0, 0}},
    {{1, 0, 0, 0}, {0, 1, -1, 1}, {1, 1, -1, 0}, {0, 0, -1, 0}},
    {{0, 1, -1, 0}, {1, 1, -1, -1}, {0, 0, -1, -1}, {1, 0, 0, -1}},
    {{1, 1, 0, -1}, {0, 0, 0, -1}, {1, 0, 1, -1}, {0, 1, 0, 0}},
};

// one thread per link (mu, parity, site): G, then F = -TA(U G) in the QDP gauge layout
__global__ void __launch_bounds__(128) force_link_kernel(const __grid_constant__ ForceArgs a,
                                                         const __grid_constant__ Spin sp) {
  const long n = 8 * a.vh;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
    const int mu = (int)(idx / (2 * a.vh));
    const int p = (int)((idx / a.vh) & 1);
    const long i = idx % a.vh;
    int c[4];
    coords_of(a, p, i, c);
    int cf[4] = {c[0], c[1], c[2], c[3]};
    cf[mu] += 1;
    int pn;
    long in;
    site_of(a, cf, pn, in);
    // hopping term: A = Y (+) W, B = X (+) Z by parity
    cd A0[12], B1[12];
    load_spinor(p == 0 ? a.Y : a.W, a.stride, i, A0);
    load_spinor(pn == 0 ? a.X : a.Z, a.stride, in, B1);
    double2 proj[4][4];
#pragma unroll
    for (int al = 0; al < 4; al++)
#pragma unroll
      for (int be = 0; be < 4; be++)
        proj[al][be] = make_double2((al == be ? 1.0 : 0.0) - sp.gam[mu][al][be].x, -sp.gam[mu][al][be].y);
    const M3 P = spin_outer(proj, B1, A0);
    cd B0[12], A1[12];
    load_spinor(p == 0 ? a.X : a.Z, a.stride, i, B0);
    load_spinor(pn == 0 ? a.Y : a.W, a.stride, in, A1);
#pragma unroll
    for (int al = 0; al < 4; al++)
#pragma unroll
      for (int be = 0; be < 4; be++)
        proj[al][be] = make_double2((al == be ? 1.0 : 0.0) + sp.gam[mu][al][be].x, sp.gam[mu][al][be].y);
    const M3 K = spin_outer(proj, B0, A1);
    const double eta = (mu == 3 && c[3] == a.dims[3] - 1) ? (double)a.tb : 1.0;
    const double hk = 2.0 * a.kappa * a.kappa * eta;
    M3 G;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
      for (int s = 0; s < 3; s++) G.m[r][s] = hk * (P.m[r][s] + conj(K.m[s][r]));
    // clover term: the leaves of the three planes that contain mu
    int pl = 0;
    for (int m = 0; m < 4; m++)
      for (int nn = m + 1; nn < 4; nn++, pl++) {
        if (m != mu && nn != mu) continue;
        const int self = (m == mu) ? 0 : 1;
        for (int lf = 0; lf < 4; lf++)
          for (int j = 0; j < 4; j++) {
            const LeafFactor fj = c_leaves[lf][j];
            if (fj.dir != self) continue;
            // the leaf's start s: the link sits at s + (om, on)
            int s0[4] = {c[0], c[1], c[2], c[3]};
            s0[m] -= fj.om;
            s0[nn] -= fj.on;
            M3 after = m3_eye(), before = m3_eye();
            for (int k = 0; k < 4; k++) {
              if (k == j) continue;
              const LeafFactor fk = c_leaves[lf][k];
              int sk[4] = {s0[0], s0[1], s0[2], s0[3]};
              sk[m] += fk.om;
              sk[nn] += fk.on;
              M3 u = load_link(a, fk.dir == 0 ? m : nn, sk);
              if (fk.dag) u = m3_dag(u);
              if (k > j)
                after = m3_mul(after, u);
              else
                before = m3_mul(before, u);
            }
            M3 r = m3_mul(m3_mul(after, load_omega(a, pl, s0)), before);
            if (fj.dag) r = m3_dag(r);
#pragma unroll
            for (int x = 0; x < 3; x++)
#pragma unroll
              for (int y = 0; y < 3; y++) G.m[x][y] = G.m[x][y] + r.m[x][y];
          }
      }
    // F = -TA(U G)
    const M3 UG = m3_mul(load_link(a, mu, c), G);
    M3 F;
    cd tr = {0.0, 0.0};
#pragma unroll
    for (int x = 0; x < 3; x++)
#pragma unroll
      for (int y = 0; y < 3; y++) F.m[x][y] = -0.5 * (UG.m[x][y] - conj(UG.m[y][x]));
#pragma unroll
    for (int x = 0; x < 3; x++) tr = tr + F.m[x][x];
#pragma unroll
    for (int x = 0; x < 3; x++) F.m[x][x] = F.m[x][x] - (1.0 / 3.0) * tr;
    double2* o = a.out + ((long)(mu * 2 + p) * a.vh + i) * 9;
#pragma unroll
    for (int k = 0; k < 9; k++) o[k] = make_double2(F.m[k / 3][k % 3].re, F.m[k / 3][k % 3].im);
  }
}

void fill_spin(Spin& sp) {
  // DeGrand-Rossi: g_x, g_y, g_z, g_t (row-major, complex)
  static const double g[4][4][4][2] = {
      {{{0, 0}, {0, 0}, {0, 0}, {0, 1}}, {{0, 0}, {0, 0}, {0, 1}, {0, 0}}, {{0, 0}, {0, -1}, {0, 0}, {0, 0}},
       {{0, -1}, {0, 0}, {0, 0}, {0, 0}}},
      {{{0, 0}, {0, 0}, {0, 0}, {-1, 0}}, {{0, 0}, {0, 0}, {1, 0}, {0, 0}}, {{0, 0}, {1, 0}, {0, 0}, {0, 0}},
       {{-1, 0}, {0, 0}, {0, 0}, {0, 0}}},
      {{{0, 0}, {0, 0}, {0, 1}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {0, -1}}, {{0, -1}, {0, 0}, {0, 0}, {0, 0}},
       {{0, 0}, {0, 1}, {0, 0}, {0, 0}}},
      {{{0, 0}, {0, 0}, {1, 0}, {0, 0}}, {{0, 0}, {0, 0}, {0, 0}, {1, 0}}, {{1, 0}, {0, 0}, {0, 0}, {0, 0}},
       {{0, 0}, {1, 0}, {0, 0}, {0, 0}}}};
  for (int m = 0; m < 4; m++)
    for (int r = 0; r < 4; r++)
      for (int s = 0; s < 4; s++) sp.gam[m][r][s] = make_double2(g[m][r][s][0], g[m][r][s][1]);
  int pl = 0;
  for (int m = 0; m < 4; m++)
    for (int nn = m + 1; nn < 4; nn++, pl++)
      for (int r = 0; r < 4; r++)
        for (int s = 0; s < 4; s++) {
          double re = 0, im = 0;
          for (int k = 0; k < 4; k++) {
            // g_m[r][k] g_n[k][s] - g_n[r][k] g_m[k][s]
            const double* a1 = g[m][r][k];
            const double* b1 = g[nn][k][s];
            const double* a2 = g[nn][r][k];
            const double* b2 = g[m][k][s];
            re += a1[0] * b1[0] - a1[1] * b1[1] - (a2[0] * b2[0] - a2[1] * b2[1]);
            im += a1[0] * b1[1] + a1[1] * b1[0] - (a2[0] * b2[1] + a2[1] * b2[0]);
          }
          sp.sig[pl][r][s] = make_double2(0.5 * re, 0.5 * im);
        }
}

int force_grid(long n) {
  long b = (n + 127) / 128;
  return (int)(b < 152L * 64 ? b : 152L * 64);
}

}  // namespace
}  // namespace wcl

using namespace wcl;

extern "C" {

wcl_status wcl_clover_force(wcl_ctx* c, void* d_force, const void* d_x_e, int include_logdet) {
  if (!c || !d_force || !d_x_e) {
    set_error("wcl_clover_force: null pointer");
    return WCL_ERR_INVALID_ARG;
  }
  if (!c->lat.loaded) {
    set_error("wcl_clover_force: no gauge field loaded");
    return WCL_ERR_NO_GAUGE;
  }
  if (!(c->lat.tw == 1.0 && c->lat.csw_t == c->lat.csw)) {
    set_error("wcl_clover_force: the force is defined for the isotropic operator (wcl_load_gauge)");
    return WCL_ERR_INVALID_ARG;
  }
  const void* xin = nullptr;
  const void* fout = nullptr;
  if (!wcl_resolve_field(c, d_x_e, &xin, "wcl_clover_force x") ||
      !wcl_resolve_field(c, d_force, &fout, "wcl_clover_force force"))
    return WCL_ERR_INVALID_ARG;
  WCL_CHECK(wcl_enter(c));
  const LatticeDevice& L = c->lat;
  std::vector<wcl_ctx*> v{c};
  FieldRef X, Y, Z, W, T;
  WCL_CHECK(ws_field(v, "F_X", F64, 1, &X));
  WCL_CHECK(ws_field(v, "F_Y", F64, 1, &Y));
  WCL_CHECK(ws_field(v, "F_Z", F64, 1, &Z));
  WCL_CHECK(ws_field(v, "F_W", F64, 1, &W));
  WCL_CHECK(ws_field(v, "F_T", F64, 1, &T));
  void* om = nullptr;
  WCL_CHECK(ws_get(c, "F_omega", sizeof(double2) * 6 * 9 * 2 * (size_t)L.vh, &om));
  WCL_CUDA(cudaMemsetAsync(c->d_flags, 0, sizeof(int), c->stream));
  WCL_CUDA(import_fermion(L, xin, L.vh * 12, 0, 1, X.ptr[0], c->d_flags, c->stream));
  count_launch(c);
  // Y = M_hat X, Z = A_oo^-1 D_oe X, W = A_oo^-1 D^+_oe Y
  WCL_CHECK(apply_mhat(v, F64, 1, Y, X, T, false, nullptr));
  WCL_CHECK(dslash(v, F64, 1, Z, X, nullptr, 1, false, CL_AINV, CL_NONE, C_ONE, C_ZERO, nullptr));
  WCL_CHECK(dslash(v, F64, 1, W, Y, nullptr, 1, true, CL_AINV, CL_NONE, C_ONE, C_ZERO, nullptr));
  ForceArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int d = 0; d < 4; d++) a.dims[d] = L.dims[d];
  a.lxh = L.dims[0] / 2;
  a.vh = L.vh;
  a.stride = L.stride;
  a.tb = L.tb;
  a.kappa = L.kappa;
  a.csw = L.csw;
  a.logdet = include_logdet ? 1 : 0;
  a.gauge[0] = static_cast<const double2*>(L.gauge[F64][0]);
  a.gauge[1] = static_cast<const double2*>(L.gauge[F64][1]);
  a.ainv_odd = static_cast<const double2*>(L.clovinv[F64][1]);
  a.X = static_cast<const double2*>(X.ptr[0]);
  a.Y = static_cast<const double2*>(Y.ptr[0]);
  a.Z = static_cast<const double2*>(Z.ptr[0]);
  a.W = static_cast<const double2*>(W.ptr[0]);
  a.omega = static_cast<double2*>(om);
  a.out = static_cast<double2*>(const_cast<void*>(fout));
  Spin sp;
  fill_spin(sp);
  force_omega_kernel<<<force_grid(2 * L.vh), 128, 0, c->stream>>>(a, sp);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  force_link_kernel<<<force_grid(8 * L.vh), 128, 0, c->stream>>>(a, sp);
  WCL_CUDA(cudaGetLastError());
  count_launch(c);
  WCL_CUDA(cudaMemcpyAsync(c->h_flags, c->d_flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  WCL_CHECK(wcl_leave(c, WCL_OK));
  if (c->h_flags[0] & 1) {
    set_error("wcl_clover_force: non-finite entry in x");
    return WCL_ERR_NONFINITE;
  }
  return WCL_OK;
}

}  // extern "C"
