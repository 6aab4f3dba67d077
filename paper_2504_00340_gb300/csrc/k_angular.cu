// k_angular.cu -- angular substep A(h) (Section 3.4, Eqs. sd and fly): the
// five-point Laplacian in (u, v) with zero Dirichlet values is diagonalised by
// the discrete sine transform (DST-I); each mode (m, n) is advanced by
// Crank-Nicolson with coefficient kappa/2, kappa = rho sigma_tr,g:
//   psi^ <- psi^ (1 + h kappa lam_mn / 4) / (1 - h kappa lam_mn / 4),
//   lam_mn = (2cos(pi m/(Nu+1)) - 2)/du^2 + (2cos(pi n/(Nv+1)) - 2)/dv^2.
// The transform is the orthonormal DST-I, sqrt(2/(N+1)) sin(pi m i/(N+1)),
// which is symmetric and its own inverse; the paper's FFT-based evaluation is
// replaced by dense 16-point sine sums folded by the (anti)symmetry
// S[m][N-1-i] = (-1)^m S[m][i], which halves the multiply-adds.
//
// GB300 design.  A CTA owns one (component, g, c) and 32 lateral points (16 in
// FP64).  Thread (x, j) loads row j of slab x straight from global memory
// (each warp load is one coalesced 128-byte row of the [angle][lateral] plane
// stack) and transforms it along u into shared memory; thread (x, m)
// transforms column m along v, scales by the mode factor, transforms back
// along v; thread (x, j) transforms back along u and stores to global memory.
// Sine and eigenvalue tables travel as kernel parameters (constant bank).
//
// FP32 forms, chosen by the autotuner: the packed forms (k_angular_f2,
// angular_form 2-6) transform two lateral points per thread on FP32x2 pairs;
// form 5, the default for FP32, holds the N/2 distinct sine magnitudes in
// registers (angular_f2.cuh).  The TMA-staged form (k_angular_tma) has a
// persistent CTA walk its tiles of [all angles x 32 lateral points] of one
// (component, g, c); each tile comes in by one 2-D TMA copy
// (cp.async.bulk.tensor, rows nyz apart in memory) into one of three
// shared-memory buffers, is transformed in place (u, then v with the mode
// factor, then u back) and leaves by one TMA store, while the next two tiles
// load.  The direct form (k_angular) serves FP64 and grids whose row pitch
// breaks the TMA rules.
#include "pbs_internal.cuh"
#include "angular_f2.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

namespace pbs {

namespace {

using namespace ang;

// lateral points per CTA: one 128-byte row of the tile per angle
template <typename real>
__host__ __device__ constexpr int tile_w() { return sizeof(real) == 8 ? 16 : 32; }

// Orthonormal DST-I matrices sqrt(2/(N+1)) sin(pi (m+1)(i+1)/(N+1)) for every
// even size N <= 16, row-major [m][i], packed one after another (size N at
// offset dst_off(N)) in the constant bank (they depend on N only).  Indexed
// with compile-time offsets, so the multiply-adds read them as constant
// operands.  The pair table of the packed FP32x2 form, c_dst_f2, is in
// angular_f2.cuh.
__constant__ float c_dst_f[kDstEntries];
__constant__ double c_dst_d[kDstEntries];

template <typename real>
struct DstTab;
template <>
struct DstTab<float> {
  template <int N>
  static __device__ __forceinline__ float at(int idx) { return c_dst_f[dst_off(N) + idx]; }
};
template <>
struct DstTab<double> {
  template <int N>
  static __device__ __forceinline__ double at(int idx) { return c_dst_d[dst_off(N) + idx]; }
};


// y[m] = sum_i S[m][i] x[i] for an orthonormal DST-I of even length N.
template <typename real, int N>
__device__ __forceinline__ void dst_apply(const real (&x)[N], real (&y)[N]) {
  constexpr int H = N / 2;
  real e[H], o[H];
#pragma unroll
  for (int i = 0; i < H; i++) {
    e[i] = x[i] + x[N - 1 - i];
    o[i] = x[i] - x[N - 1 - i];
  }
#pragma unroll
  for (int m = 0; m < N; m++) y[m] = 0;
#pragma unroll
  for (int i = 0; i < H; i++)
#pragma unroll
    for (int m = 0; m < N; m++) y[m] = fma(DstTab<real>::template at<N>(m * N + i), (m & 1) ? o[i] : e[i], y[m]);
}

template <typename real, int NU, int NV, bool EXACT>
__global__ void __launch_bounds__(tile_w<real>() * (NU > NV ? NU : NV), 2)
    k_angular(real *__restrict__ psi, const real *__restrict__ rho_yz, const real *__restrict__ ts, int nyz,
              int ng, real hq, long long kgc0, const __grid_constant__ AngTables<real> tb) {
  constexpr int NA = NU * NV;
  constexpr int kTW = tile_w<real>();
  __shared__ real tile[NA][kTW];
  const int x = threadIdx.x;
  const int t = threadIdx.y;
  const long long kgc = kgc0 + blockIdx.y;  // (k * ng + g) * 2 + c
  const int g = (int)((kgc / 2) % ng);
  const int yz0 = blockIdx.x * kTW;
  const int yz = yz0 + x;
  const bool active = yz < nyz;
  real *base = psi + kgc * (long long)NA * nyz + yz;

  constexpr int NT = NU > NV ? NU : NV;
  // forward transform along u: thread row t < NV loads row j = t of its slab
  // straight from global memory (coalesced over the 32 lateral points)
  if (t < NV) {
    real r[NU], y[NU];
#pragma unroll
    for (int i = 0; i < NU; i++) r[i] = active ? base[(long long)(t * NU + i) * nyz] : real(0);
    dst_apply<real, NU>(r, y);
#pragma unroll
    for (int i = 0; i < NU; i++) tile[t * NU + i][x] = y[i];
  }
  __syncthreads();
  // along v: forward, mode factor, inverse (column m = t)
  if (t < NU) {
    const real q = active ? hq * rho_yz[yz] * ts[g] : real(0);  // h kappa / 4
    real c[NV], y[NV];
#pragma unroll
    for (int j = 0; j < NV; j++) c[j] = tile[j * NU + t][x];
    dst_apply<real, NV>(c, y);
#pragma unroll
    for (int n = 0; n < NV; n++) y[n] *= mode_scale<EXACT>(q * tb.lam[n * NU + t]);  // lam <= 0
    dst_apply<real, NV>(y, c);
#pragma unroll
    for (int j = 0; j < NV; j++) tile[j * NU + t][x] = c[j];
  }
  __syncthreads();
  // inverse along u and store
  if (t < NV) {
    real r[NU], y[NU];
#pragma unroll
    for (int i = 0; i < NU; i++) r[i] = tile[t * NU + i][x];
    dst_apply<real, NU>(r, y);
    if (active) {
#pragma unroll
      for (int i = 0; i < NU; i++) base[(long long)(t * NU + i) * nyz] = y[i];
    }
  }
  (void)NT;
}

// ---------------------------------------------------------------- packed FP32 form

// MINB > 0: registers capped so that MINB CTAs fit an SM (more warps to hide
// the load latency).  PAIR: each CTA takes two consecutive slab stacks, the
// second's rows asked of the L2 while the first is transformed.  REGC: the
// sine coefficients from registers (N/2 magnitudes per size, signs known at
// compile time) instead of constant-bank pairs, each of which costs a move.
template <int NU, int NV, bool EXACT, int MINB, bool PAIR, bool REGC = false>
__global__ void __launch_bounds__(kF2X * (NU > NV ? NU : NV), MINB)
    k_angular_f2(float *__restrict__ psi, const float *__restrict__ rho_yz, const float *__restrict__ ts, int nyz,
                 int ng, float hq, long long kgc0, long long kgc_end, const __grid_constant__ AngTables<float> tb) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if constexpr (PAIR) {
    const long long k = kgc0 + 2 * (long long)blockIdx.y;
    if (k + 1 < kgc_end && threadIdx.x == 0 && threadIdx.y < NV) {
      const int yz = blockIdx.x * kF2X * 2;
      const float *base = psi + (k + 1) * (long long)(NU * NV) * nyz + yz;
#pragma unroll
      for (int i = 0; i < NU; i++)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (long long)(threadIdx.y * NU + i) * nyz));
    }
    angular_f2_tile<NU, NV, EXACT, REGC>(psi, rho_yz, ts, nyz, ng, hq, k, blockIdx.x, threadIdx.x, threadIdx.y,
                                         smem_raw, tb);
    if (k + 1 < kgc_end) {
      __syncthreads();  // the tile is reused
      angular_f2_tile<NU, NV, EXACT, REGC>(psi, rho_yz, ts, nyz, ng, hq, k + 1, blockIdx.x, threadIdx.x, threadIdx.y,
                                           smem_raw, tb);
    }
  } else {
    angular_f2_tile<NU, NV, EXACT, REGC>(psi, rho_yz, ts, nyz, ng, hq, kgc0 + blockIdx.y, blockIdx.x, threadIdx.x,
                                         threadIdx.y, smem_raw, tb);
  }
}

template <int NU, int NV, bool EXACT, int MINB, bool PAIR, bool REGC = false>
cudaError_t go_f2_form(const LaunchCtx &lc, const Dims &d, float *psi, const float *rho_yz, const float *ts, double h,
                       const AngTables<float> &tb) {
  constexpr int NT = NU > NV ? NU : NV;
  auto kern = k_angular_f2<NU, NV, EXACT, MINB, PAIR, REGC>;
  const size_t smem = sizeof(float2) * NU * NV * kF2X;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long total = (long long)d.ncomp * d.ng * 2;
  const long long per = PAIR ? 2 : 1;  // slab stacks per CTA
  for (long long k0 = 0; k0 < total; k0 += 65535 * per) {
    const long long cnt = std::min(total - k0, 65535 * per);
    dim3 grid((d.nyz / 2 + kF2X - 1) / kF2X, (unsigned)((cnt + per - 1) / per));
    kern<<<grid, dim3(kF2X, NT), smem, lc.stream>>>(psi, rho_yz, ts, d.nyz, d.ng, (float)(0.25 * h), k0, k0 + cnt, tb);
    ++*lc.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Packed FP32 forms (angular_form 2, 3, 4; 5, 6 and 7 with the coefficients
// in registers: as compiled, capped at 85 registers, two stacks per CTA).
template <int NU, int NV, bool EXACT>
cudaError_t go_f2(const LaunchCtx &lc, const Dims &d, float *psi, const float *rho_yz, const float *ts, double h,
                  const AngTables<float> &tb) {
  constexpr int NT = NU > NV ? NU : NV;
  constexpr int kMinB = 1024 / (kF2X * NT);  // 64 registers per thread
  constexpr int kMinB3 = 768 / (kF2X * NT);  // 85 registers per thread
  if (lc.angular_form == 5) return go_f2_form<NU, NV, EXACT, 0, false, true>(lc, d, psi, rho_yz, ts, h, tb);
  if (lc.angular_form == 6) return go_f2_form<NU, NV, EXACT, kMinB3, false, true>(lc, d, psi, rho_yz, ts, h, tb);
  if (lc.angular_form == 7) return go_f2_form<NU, NV, EXACT, 0, true, true>(lc, d, psi, rho_yz, ts, h, tb);
  if (lc.angular_form == 3) return go_f2_form<NU, NV, EXACT, kMinB, false>(lc, d, psi, rho_yz, ts, h, tb);
  if (lc.angular_form == 4) return go_f2_form<NU, NV, EXACT, 0, true>(lc, d, psi, rho_yz, ts, h, tb);
  return go_f2_form<NU, NV, EXACT, 0, false>(lc, d, psi, rho_yz, ts, h, tb);
}

// ---------------------------------------------------------------- TMA form

constexpr int kAngBufs = 3;                        // tiles in flight per CTA
constexpr long long kAngWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bounded waits

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(x),
               "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Tile t covers rows [stack * NA, stack * NA + NA) and lateral points
// [tx * TW, tx * TW + TW) with stack = t / ntx (= (k * ng + g) * 2 + c).
template <typename real, int NU, int NV, bool EXACT>
__global__ void __launch_bounds__(tile_w<real>() * (NU > NV ? NU : NV), 2)
    k_angular_tma(const __grid_constant__ CUtensorMap map, const real *__restrict__ rho_yz,
                  const real *__restrict__ ts, int nyz, int ng, int ntx, long long ntiles, real hq,
                  const __grid_constant__ AngTables<real> tb, int *err) {
  constexpr int NA = NU * NV;
  constexpr int kTW = tile_w<real>();
  constexpr unsigned kTileBytes = NA * kTW * sizeof(real);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real(*buf)[NA][kTW] = reinterpret_cast<real(*)[NA][kTW]>(smem_raw);
  __shared__ __align__(8) uint64_t full[kAngBufs];
  const int x = threadIdx.x, t = threadIdx.y;
  const bool leader = (x == 0 && t == 0);
  const long long step = gridDim.x;
  if (leader) {
    for (int b = 0; b < kAngBufs; b++) mbar_init(&full[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // prologue: the CTA's first kAngBufs - 1 tiles
  if (leader) {
    for (int j = 0; j < kAngBufs - 1; j++) {
      const long long tile = blockIdx.x + j * step;
      if (tile < ntiles) {
        mbar_arrive_expect_tx(&full[j], kTileBytes);
        tma_load_2d(buf[j], &map, (int)(tile % ntx) * kTW, (int)(tile / ntx) * NA, &full[j]);
      }
    }
  }
  long long i = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += step, i++) {
    const int b = (int)(i % kAngBufs);
    const bool ok = mbar_wait_bounded(&full[b], (unsigned)((i / kAngBufs) & 1), kAngWaitCycles);
    if (__syncthreads_or(!ok)) {
      // a copy never arrived: record it, let the copies in flight land, stop
      if (leader) {
        atomicAdd(err, 1);
        err[1] = kErrTimeoutAngular;
        for (int j = 1; j < kAngBufs; j++) {
          const long long ti = tile + j * step;
          if (ti < ntiles && j < kAngBufs - 1)
            mbar_wait_bounded(&full[(b + j) % kAngBufs], (unsigned)(((i + j) / kAngBufs) & 1), kAngWaitCycles);
        }
        bulk_wait_all();
      }
      return;
    }
    real(*tl)[kTW] = buf[b];
    const long long stack = tile / ntx;
    const int g = (int)((stack / 2) % ng);
    const int yz = (int)(tile % ntx) * kTW + x;
    constexpr int NT = NU > NV ? NU : NV;
    // along u: row t of the slab, in place
    if (t < NV) {
      real r[NU], y[NU];
#pragma unroll
      for (int k = 0; k < NU; k++) r[k] = tl[t * NU + k][x];
      dst_apply<real, NU>(r, y);
#pragma unroll
      for (int k = 0; k < NU; k++) tl[t * NU + k][x] = y[k];
    }
    __syncthreads();
    // along v with the mode factor: column m = t
    if (t < NU) {
      const real q = (yz < nyz) ? hq * rho_yz[yz] * ts[g] : real(0);  // h kappa / 4
      real c[NV], y[NV];
#pragma unroll
      for (int j = 0; j < NV; j++) c[j] = tl[j * NU + t][x];
      dst_apply<real, NV>(c, y);
#pragma unroll
      for (int n = 0; n < NV; n++) y[n] *= mode_scale<EXACT>(q * tb.lam[n * NU + t]);
      dst_apply<real, NV>(y, c);
#pragma unroll
      for (int j = 0; j < NV; j++) tl[j * NU + t][x] = c[j];
    }
    __syncthreads();
    // back along u
    if (t < NV) {
      real r[NU], y[NU];
#pragma unroll
      for (int k = 0; k < NU; k++) r[k] = tl[t * NU + k][x];
      dst_apply<real, NU>(r, y);
#pragma unroll
      for (int k = 0; k < NU; k++) tl[t * NU + k][x] = y[k];
    }
    fence_proxy_async_smem();  // the generic-proxy writes become visible to the TMA store
    __syncthreads();
    if (leader) {
      tma_store_2d(&map, (int)(tile % ntx) * kTW, (int)stack * NA, tl);
      bulk_commit();
      // buffer of tile i + kAngBufs - 1 last held tile i - 1: its store must have read it
      const long long nt = tile + (kAngBufs - 1) * step;
      if (nt < ntiles) {
        bulk_wait_read<1>();
        const int nb = (int)((i + kAngBufs - 1) % kAngBufs);
        mbar_arrive_expect_tx(&full[nb], kTileBytes);
        tma_load_2d(buf[nb], &map, (int)(nt % ntx) * kTW, (int)(nt / ntx) * NA, &full[nb]);
      }
    }
    (void)NT;
  }
  if (leader) bulk_wait_all();
}

// TMA form usable: row pitch nyz * sizeof(real) a multiple of 16 bytes, rows
// addressable by 32-bit coordinates, and the driver's encoder available.
template <typename real>
bool angular_tma_ok(const Dims &d, const real *psi) {
  const long long rows = (long long)d.ncomp * d.ng * 2 * d.na;
  return ((d.nyz * sizeof(real)) % 16 == 0) && rows < (1LL << 31) && d.na <= 256 &&
         (reinterpret_cast<uintptr_t>(psi) % 16 == 0) && tensor_map_encoder() != nullptr;
}

template <typename real, int NU, int NV, bool EXACT>
cudaError_t go_tma(const LaunchCtx &lc, const Dims &d, real *psi, const real *rho_yz, const real *ts, double h,
                   const AngTables<real> &tb) {
  constexpr int NA = NU * NV;
  constexpr int kTW = tile_w<real>();
  constexpr int NT = NU > NV ? NU : NV;
  const long long rows = (long long)d.ncomp * d.ng * 2 * NA;
  CUtensorMap map;
  cuuint64_t dims[2] = {(cuuint64_t)d.nyz, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)d.nyz * sizeof(real)};
  cuuint32_t box[2] = {(cuuint32_t)kTW, (cuuint32_t)NA};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = tensor_map_encoder()(&map, sizeof(real) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           2, psi, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int ntx = (d.nyz + kTW - 1) / kTW;
  const long long ntiles = rows / NA * ntx;
  const size_t smem = (size_t)kAngBufs * NA * kTW * sizeof(real);
  auto kern = k_angular_tma<real, NU, NV, EXACT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTW * NT, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = (long long)per_sm * lc.num_sms;
  if (blocks > ntiles) blocks = ntiles;
  kern<<<(unsigned)blocks, dim3(kTW, NT), smem, lc.stream>>>(map, rho_yz, ts, d.nyz, d.ng, ntx, ntiles,
                                                               (real)(0.25 * h), tb, lc.err);
  ++*lc.launches;
  return cudaGetLastError();
}

template <typename real, int NU, int NV, bool EXACT>
cudaError_t go_exact(const LaunchCtx &lc, const Dims &d, real *psi, const real *rho_yz, const real *ts, double h,
                     const AngTables<real> &tb) {
  if constexpr (sizeof(real) == 4) {
    if (lc.angular_form >= 2 && (d.nyz % 2) == 0) return go_f2<NU, NV, EXACT>(lc, d, psi, rho_yz, ts, h, tb);
  }
  if (lc.angular_form == 1 && lc.err && angular_tma_ok<real>(d, psi))
    return go_tma<real, NU, NV, EXACT>(lc, d, psi, rho_yz, ts, h, tb);
  constexpr int NT = NU > NV ? NU : NV;
  constexpr int kTW = tile_w<real>();
  dim3 block(kTW, NT);
  // grid.y is limited to 65535 slab stacks per launch: larger batches go in chunks
  const long long total = (long long)d.ncomp * d.ng * 2;
  for (long long k0 = 0; k0 < total; k0 += 65535) {
    const long long cnt = total - k0 < 65535 ? total - k0 : 65535;
    dim3 grid((d.nyz + kTW - 1) / kTW, (unsigned)cnt);
    k_angular<real, NU, NV, EXACT><<<grid, block, 0, lc.stream>>>(psi, rho_yz, ts, d.nyz, d.ng, (real)(0.25 * h), k0,
                                                                   tb);
    ++*lc.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename real, int NU, int NV>
cudaError_t go(const LaunchCtx &lc, const Dims &d, real *psi, const real *rho_yz, const real *ts, double h, double du,
               double dv) {
  AngTables<real> tb;
  fill_tables(tb, NU, NV, du, dv);
  if (lc.angular_exact) return go_exact<real, NU, NV, true>(lc, d, psi, rho_yz, ts, h, tb);
  return go_exact<real, NU, NV, false>(lc, d, psi, rho_yz, ts, h, tb);
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <typename real>
cudaError_t launch_angular(const LaunchCtx &lc, const Dims &d, real *psi, const real *rho_yz, const real *ts,
                           double h, double du, double dv) {
#define PBS_ANG(A, B) \
  if (d.nu == A && d.nv == B) return go<real, A, B>(lc, d, psi, rho_yz, ts, h, du, dv);
  PBS_ANG(2, 2) PBS_ANG(4, 4) PBS_ANG(6, 6) PBS_ANG(8, 8) PBS_ANG(10, 10) PBS_ANG(12, 12) PBS_ANG(14, 14)
  PBS_ANG(16, 16) PBS_ANG(4, 8) PBS_ANG(8, 4) PBS_ANG(8, 16) PBS_ANG(16, 8) PBS_ANG(6, 4) PBS_ANG(4, 6)
#undef PBS_ANG
  return cudaErrorNotSupported;
}

cudaError_t angular_init_tables() {
  static float hf[kDstEntries];
  static double hd[kDstEntries];
  const double pi = 3.14159265358979323846;
  for (int n = 2; n <= kMaxAngle; n += 2)
    for (int m = 0; m < n; m++)
      for (int i = 0; i < n; i++) {
        const double v = std::sqrt(2.0 / (n + 1)) * std::sin(pi * (m + 1) * (i + 1) / (n + 1));
        const int at = dst_off(n) + m * n + i;
        hd[at] = v;
        hf[at] = (float)v;
      }
  cudaError_t e = cudaMemcpyToSymbol(c_dst_f, hf, sizeof(hf));
  if (e != cudaSuccess) return e;
  if ((e = upload_dst_f2()) != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_dst_d, hd, sizeof(hd));
}

bool angular_supported(int nu, int nv) {
  static const int ok[][2] = {{2, 2}, {4, 4}, {6, 6}, {8, 8}, {10, 10}, {12, 12}, {14, 14}, {16, 16},
                              {4, 8}, {8, 4}, {8, 16}, {16, 8}, {6, 4}, {4, 6}};
  for (auto &p : ok)
    if (p[0] == nu && p[1] == nv) return true;
  return false;
}

template cudaError_t launch_angular<double>(const LaunchCtx &, const Dims &, double *, const double *, const double *,
                                            double, double, double);
template cudaError_t launch_angular<float>(const LaunchCtx &, const Dims &, float *, const float *, const float *,
                                           double, double, double);

}  // namespace pbs
