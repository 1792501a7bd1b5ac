// Multi-RHS FP32 fused dslash + clover with the tile's links and clover brought into
// shared memory by the Tensor Memory Accelerator (cp.async.bulk.tensor), double buffered
// in a persistent CTA.
//
// Same operator, modes and per-thread arithmetic as dslash_mrhs_kernel (one thread per
// (site, RHS), links with row 2 rebuilt and clover unpacked once per tile for all
// right-hand sides).  What changes is how the tile's links and clover arrive: a tile is
// one whole x-row of output sites (Lx/2 = 16 sites: the variant applies when Lx = 32),
// so that every set it needs is one contiguous run of every chunk row --
//   the 8 x 3 forward link chunks at the row           (one 64 x 12 float box),
//   the 3 backward link chunks of each direction mu at the row one step back in mu
//   (for mu = x the same row of the other parity)      (four 64 x 3 boxes),
//   the 18 clover chunks at the row                     (one 64 x 18 box) --
// and one thread issues these six tensor copies for the NEXT tile into the other stage
// while the CTA computes the current one; an mbarrier with the expected byte count
// tells the CTA when a stage has landed.  The copies go global -> shared memory
// without registers or load instructions, so the DRAM latency of the staging leaves
// the per-tile critical path.  Every wait on an mbarrier is bounded: on expiry the CTA
// records the failure in `err` and stops.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "blackwell.cuh"
#include "context.cuh"

namespace wcl {

constexpr int TMA_TS = 16;                          // sites per tile = Lx / 2
constexpr int TMA_FWD_BYTES = 12 * 64 * 4;          // 12 chunk rows x 64 floats
constexpr int TMA_BWD_BYTES = 3 * 64 * 4;           // per direction
constexpr int TMA_CLOV_BYTES = 18 * 64 * 4;
constexpr int TMA_STAGE_BYTES = TMA_FWD_BYTES + 4 * TMA_BWD_BYTES + TMA_CLOV_BYTES;  // 10752
constexpr long TMA_WAIT_LIMIT = 1L << 24;           // try_wait polls before giving up

struct TmaMaps {
  CUtensorMap fwd;   // links of the output parity, box 64 x 12
  CUtensorMap bwd;   // links of the other parity, box 64 x 3
  CUtensorMap clov;  // clover of the output parity (post or pre), box 64 x 18
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

struct TmaRow {
  int y, z, t;
};
__device__ __forceinline__ TmaRow tma_row(const LatGeom& g, long row) {
  TmaRow r;
  r.y = (int)(row % g.dims[1]);
  long q = row / g.dims[1];
  r.z = (int)(q % g.dims[2]);
  r.t = (int)(q / g.dims[2]);
  return r;
}
__device__ __forceinline__ long tma_row_index(const LatGeom& g, int y, int z, int t) {
  return ((long)t * g.dims[2] + z) * g.dims[1] + y;
}

// the six tensor copies of tile `row` into a stage
__device__ __forceinline__ void tma_issue(const TmaMaps& m, const LatGeom& g, long row, float* stage, uint64_t* bar) {
  const TmaRow r = tma_row(g, row);
  const int yb = r.y == 0 ? g.dims[1] - 1 : r.y - 1;
  const int zb = r.z == 0 ? g.dims[2] - 1 : r.z - 1;
  const int tb = r.t == 0 ? g.dims[3] - 1 : r.t - 1;
  const long rows_b[4] = {row, tma_row_index(g, yb, r.z, r.t), tma_row_index(g, r.y, zb, r.t),
                          tma_row_index(g, r.y, r.z, tb)};
  mbar_expect_tx(bar, TMA_STAGE_BYTES);
  tma_load_2d(stage, &m.fwd, (int)(row * TMA_TS * 4), 0, bar);
  for (int mu = 0; mu < 4; mu++)
    tma_load_2d(stage + (TMA_FWD_BYTES + mu * TMA_BWD_BYTES) / 4, &m.bwd, (int)(rows_b[mu] * TMA_TS * 4), 3 * mu, bar);
  tma_load_2d(stage + (TMA_FWD_BYTES + 4 * TMA_BWD_BYTES) / 4, &m.clov, (int)(row * TMA_TS * 4), 0, bar);
}

template <bool DAG, int MODE, int EPI>
__global__ void __launch_bounds__(256, 4)
    dslash_tma_kernel(const __grid_constant__ DslashArgs a, const __grid_constant__ TmaMaps maps, int* err) {
  using R = float;
  constexpr int LROW = SmemRow<R>::LINK, CROW = SmemRow<R>::CLOV;
  __shared__ __align__(128) float raw[2][TMA_STAGE_BYTES / 4];
  __shared__ __align__(16) R Us[8][TMA_TS][LROW];
  __shared__ __align__(16) R Cs[TMA_TS][CROW];
  __shared__ int Nb[8][TMA_TS];
  __shared__ unsigned char Tb[TMA_TS];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int abort_flag;
  const LatGeom& g = a.b.lat[0];
  const R alpha = R(a.alpha[0]), beta = R(a.beta[0]);
  const int nrhs = a.nrhs_tc;
  const int p = a.out_parity;
  const long stride = g.stride;
  const long nrows = g.vh / TMA_TS;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    abort_flag = 0;
    fence_proxy_async();  // the barriers' initialisation is visible to the copy engine
  }
  __syncthreads();
  long row = blockIdx.x;
  if (threadIdx.x == 0 && row < nrows) tma_issue(maps, g, row, raw[0], &bar[0]);
  for (int it = 0; row < nrows; it++, row += gridDim.x) {
    const int st = it & 1;
    const long next = row + gridDim.x;
    if (threadIdx.x == 0 && next < nrows) {
      fence_proxy_async();  // the stage being refilled was last read by ordinary loads
      tma_issue(maps, g, next, raw[st ^ 1], &bar[st ^ 1]);
    }
    const long site0 = row * TMA_TS;
    if (threadIdx.x < TMA_TS) {
      const SiteNbr n = site_neighbours(g, p, site0 + threadIdx.x);
#pragma unroll
      for (int mu = 0; mu < 4; mu++) {
        Nb[2 * mu][threadIdx.x] = (int)n.jf[mu];
        Nb[2 * mu + 1][threadIdx.x] = (int)n.jb[mu];
      }
      Tb[threadIdx.x] = (n.t + 1 == g.dims[3] ? 1 : 0) | (n.t == 0 ? 2 : 0);
    }
    // wait for this tile's stage (phase parity = how often the stage was used before)
    bool ok = false;
    for (long k = 0; k < TMA_WAIT_LIMIT && !ok; k++) ok = mbar_try_wait(&bar[st], (it >> 1) & 1);
    if (!ok) abort_flag = 1;
    __syncthreads();
    if (abort_flag) {
      if (threadIdx.x == 0) atomicOr(err, 0x100);
      // let the copies already issued land before the CTA's shared memory is released
      for (long k = 0; k < TMA_WAIT_LIMIT; k++)
        if (mbar_try_wait(&bar[st ^ 1], ((it + 1) >> 1) & 1)) break;
      return;
    }
    // unpack: links with row 2 rebuilt, clover as rows of reals
    const float4* rs = reinterpret_cast<const float4*>(raw[st]);
    const long rowb_x = row * TMA_TS;  // the backward x links: same row of the other parity
    for (int e = threadIdx.x; e < 8 * TMA_TS; e += blockDim.x) {
      const int ls = e % TMA_TS, d = e / TMA_TS, mu = d >> 1;
      const float4* src;
      int li;
      if (d & 1) {
        src = rs + (TMA_FWD_BYTES + mu * TMA_BWD_BYTES) / 16;
        li = mu == 0 ? (int)(Nb[d][ls] - rowb_x) : ls;
      } else {
        src = rs + mu * 3 * TMA_TS;
        li = ls;
      }
      const float4 q0 = src[li], q1 = src[TMA_TS + li], q2 = src[2 * TMA_TS + li];
      cpx<R> u[3][3];
      u[0][0] = {q0.x, q0.y};
      u[0][1] = {q0.z, q0.w};
      u[0][2] = {q1.x, q1.y};
      u[1][0] = {q1.z, q1.w};
      u[1][1] = {q2.x, q2.y};
      u[1][2] = {q2.z, q2.w};
      reconstruct_row2(u);
      // the factors shared by all RHS, folded in as in dslash_mrhs_kernel: alpha into the
      // links (XPAY) or the clover term (POST), the t-hop weights into the t links
      R f = (MODE & MODE_POST) ? R(1) : alpha;
      if (d >= 6) f = f * hop_t_weight<R>(g, (Tb[ls] & (d == 6 ? 1 : 2)) != 0);
#pragma unroll
      for (int k = 0; k < 9; k++) {
        Us[d][ls][2 * k] = f * u[k / 3][k % 3].re;
        Us[d][ls][2 * k + 1] = f * u[k / 3][k % 3].im;
      }
    }
    const float4* cs = rs + (TMA_FWD_BYTES + 4 * TMA_BWD_BYTES) / 16;
    const R cf = (MODE & MODE_POST) ? alpha : beta;  // beta: the clover term applied to x
    for (int e = threadIdx.x; e < 18 * TMA_TS; e += blockDim.x) {
      const int ls = e % TMA_TS, k = e / TMA_TS;
      const float4 v = cs[k * TMA_TS + ls];
      Cs[ls][4 * k] = cf * v.x;
      Cs[ls][4 * k + 1] = cf * v.y;
      Cs[ls][4 * k + 2] = cf * v.z;
      Cs[ls][4 * k + 3] = cf * v.w;
    }
    __syncthreads();
    // compute: thread = (site ls, rhs), as in dslash_mrhs_kernel
    const int ls = threadIdx.x % TMA_TS, rhs = threadIdx.x / TMA_TS;
    const long i = site0 + ls;
    double red[3] = {0.0, 0.0, 0.0};
    const bool valid = rhs < nrhs && (!a.active || a.active[rhs]);
    if (valid) {
      const void* in = rhs_ptr<F32>(a.in, 0, rhs, stride);
      cpx<R> acc[12];
#pragma unroll
      for (int k = 0; k < 12; k++) acc[k] = {R(0), R(0)};
      const R sf = R(1), sb = R(1);  // in the staged t links
      hop_dir_smem<F32, 0, DAG>(acc, in, nullptr, stride, Nb[0][ls], Nb[1][ls], Us[0][ls], Us[1][ls], R(1), R(1));
      hop_dir_smem<F32, 1, DAG>(acc, in, nullptr, stride, Nb[2][ls], Nb[3][ls], Us[2][ls], Us[3][ls], R(1), R(1));
      hop_dir_smem<F32, 2, DAG>(acc, in, nullptr, stride, Nb[4][ls], Nb[5][ls], Us[4][ls], Us[5][ls], R(1), R(1));
      hop_dir_smem<F32, 3, DAG>(acc, in, nullptr, stride, Nb[6][ls], Nb[7][ls], Us[6][ls], Us[7][ls], sf, sb);
      if (MODE & MODE_XPAY) {
        cpx<R> xv[12];
        SpinorIO<F32>::load_cs(xv, rhs_ptr<F32>(a.x, 0, rhs, stride), nullptr, stride, i);
        hermitian6_axpy_row(acc, R(1), Cs[ls], xv);
        hermitian6_axpy_row(acc + 6, R(1), Cs[ls] + 36, xv + 6);
        if (EPI == EPI_ALPHA) {
          cpx<R> fv[12];
          SpinorIO<F32>::load_cs(fv, rhs_ptr<F32>(a.f, 0, rhs, stride), nullptr, stride, i);
          dot_acc(red, fv, acc);
        } else if (EPI == EPI_OMEGA) {
          dot_acc(red, acc, xv);
          red[2] += norm_site(acc);
        } else if (EPI == EPI_CGALPHA || EPI == EPI_CGZ) {
          red[0] += norm_site(acc);
        }
      }
      if (MODE & MODE_POST) {
        cpx<R> y2[12];
        clover_apply_smem<R>(y2, acc, Cs[ls]);
        SpinorIO<F32>::template store<true>(y2, rhs_ptr_w<F32>(a.out, 0, rhs, stride), nullptr, stride, i);
      } else {
        SpinorIO<F32>::template store<true>(acc, rhs_ptr_w<F32>(a.out, 0, rhs, stride), nullptr, stride, i);
      }
    }
    if constexpr (EPI != EPI_NONE) {
#pragma unroll
      for (int k = 0; k < 3; k++)
#pragma unroll
        for (int o = TMA_TS / 2; o; o >>= 1) red[k] += __shfl_xor_sync(0xffffffffu, red[k], o);
      if (ls == 0 && rhs < nrhs) {
        double* dst = a.partials + ((size_t)rhs * a.maxch + row) * 3;
        dst[0] = red[0];
        dst[1] = red[1];
        dst[2] = red[2];
      }
    }
    __syncthreads();  // the tile's shared rows and this stage are free for the next refill
  }
}

// ---------------------------------------------------------------------------
// host side

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled g_encode = nullptr;
std::once_flag g_encode_once;

EncodeTiled encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiled>(fn);
    else
      cudaGetLastError();
  });
  return g_encode;
}

// 2D FP32 tensor: `rows` chunk rows of 4 * stride floats, box 64 floats x box_rows
bool make_map(CUtensorMap* m, const void* base, long stride, int rows, int box_rows) {
  EncodeTiled enc = encoder();
  if (!enc || !base) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(4 * stride), (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(16 * stride)};
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

bool tma_eligible(const LatGeom& g, int nrhs) {
  return g.lxh == TMA_TS && nrhs >= 1 && nrhs <= 16 && g.vh % TMA_TS == 0 && encoder() != nullptr;
}

#define WCL_TMA_CASE(DAG, MODE, EPI)                                                              \
  case (MODE) | ((DAG) ? 16 : 0) | ((EPI) << 5):                                                 \
    dslash_tma_kernel<DAG, MODE, EPI><<<grid, threads, 0, st>>>(a, maps, err);                   \
    fin = EPI;                                                                                   \
    break;

// a.b must describe one lattice with tiles of 16 sites (one x-row each); persistent: five
// CTAs per SM walking the rows with the next row's copies in flight, else one CTA per row
// (its copies issued at its start, no overlap within the CTA)
cudaError_t launch_dslash_tma(const DslashArgs& a, bool dagger, int mode, cudaStream_t st, int* err, bool persistent) {
  const LatGeom& g = a.b.lat[0];
  if (a.b.nlat != 1 || !tma_eligible(g, a.nrhs_tc)) return cudaErrorInvalidValue;
  const int p = a.out_parity;
  const void* clov = (mode & MODE_POST) ? a.cpost[0] : a.cpre[0];
  TmaMaps maps;
  if (!make_map(&maps.fwd, a.gauge[0][p], g.stride, 12, 12) || !make_map(&maps.bwd, a.gauge[0][1 - p], g.stride, 12, 3) ||
      !make_map(&maps.clov, clov, g.stride, 18, 18))
    return cudaErrorInvalidValue;
  const int threads = (TMA_TS * a.nrhs_tc + 31) / 32 * 32;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long nrows = g.vh / TMA_TS;
  const int grid = persistent ? (int)std::min<long>(nrows, (long)nsm * 5) : (int)nrows;
  int fin = 0;
  switch (mode | (dagger ? 16 : 0)) {
    WCL_TMA_CASE(false, MODE_POST, EPI_NONE)
    WCL_TMA_CASE(true, MODE_POST, EPI_NONE)
    WCL_TMA_CASE(false, MODE_XPAY | MODE_PRE, EPI_NONE)
    WCL_TMA_CASE(true, MODE_XPAY | MODE_PRE, EPI_NONE)
    WCL_TMA_CASE(false, MODE_XPAY | MODE_PRE, EPI_ALPHA)
    WCL_TMA_CASE(false, MODE_XPAY | MODE_PRE, EPI_OMEGA)
    WCL_TMA_CASE(false, MODE_XPAY | MODE_PRE, EPI_CGALPHA)
    WCL_TMA_CASE(true, MODE_XPAY | MODE_PRE, EPI_CGZ)
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_epi_finalize(fin, a, st);
}

}  // namespace wcl
