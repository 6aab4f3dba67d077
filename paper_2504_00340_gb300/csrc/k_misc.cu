// k_misc.cu -- beam initialisation, fluence reduction and the CUDA-core form
// of the catastrophic-source angle contraction.
#include "pbs_internal.cuh"

namespace pbs {

namespace {

// psi_p(x = 0) of Eq. (bdy) as a separable product of the host-computed FP64
// projections: fe[g][c] (DG energy), fa[a] (angle cell averages), fy[p], fz[q].
// grid.y = g*2 + c (row), grid.x covers the row's na*nyz lanes; the product is
// formed in the working precision.
template <typename real>
__global__ void k_init(real *__restrict__ psi0, const double *__restrict__ fe, const double *__restrict__ fa,
                       const double *__restrict__ fy, const double *__restrict__ fz, Dims d) {
  // blockIdx.y = row (g, c), blockIdx.x = angle; the block walks the lateral points
  const int row = blockIdx.y, a = blockIdx.x;
  const real f = (real)(fe[row] * fa[a]);
  real *out = psi0 + (long long)row * d.lanes + (long long)a * d.nyz;
  for (int yz = threadIdx.x; yz < d.nyz; yz += blockDim.x) {
    const int p = yz / d.nz;
    const int q = yz - p * d.nz;
    out[yz] = f * (real)fy[p] * (real)fz[q];
  }
}

// The same product with the lateral factors converted once per block into
// shared memory (ny + nz values) and the lateral points walked row by row:
// no division and no FP64 conversion per element.  Same arithmetic order.
template <typename real>
__global__ void k_init_rows(real *__restrict__ psi0, const double *__restrict__ fe, const double *__restrict__ fa,
                            const double *__restrict__ fy, const double *__restrict__ fz, Dims d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  real *sy = reinterpret_cast<real *>(smem_raw);
  real *sz = sy + d.ny;
  for (int i = threadIdx.x; i < d.ny; i += blockDim.x) sy[i] = (real)fy[i];
  for (int i = threadIdx.x; i < d.nz; i += blockDim.x) sz[i] = (real)fz[i];
  __syncthreads();
  const int row = blockIdx.y, a = blockIdx.x;
  const real f = (real)(fe[row] * fa[a]);
  real *out = psi0 + (long long)row * d.lanes + (long long)a * d.nyz;
  for (int p = 0; p < d.ny; p++) {
    const real fp = f * sy[p];
    for (int q = threadIdx.x; q < d.nz; q += blockDim.x) out[p * d.nz + q] = fp * sz[q];
  }
}

// Planar fluence of the current state: flu[yz] += scale * sum_{k,g,a} dE_g psi^1
// (one thread per (yz, a); the sum over k and g in the working precision).
template <typename real>
__global__ void k_fluence(const real *__restrict__ psi, int ncomp_beam, const GroupCoef<real> *__restrict__ coef,
                          double *flu, Dims d, double scale) {
  const int yz = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y;
  if (yz >= d.nyz) return;
  real acc = 0;
  const real *p = psi + (long long)a * d.nyz + yz;
  for (int k = 0; k < ncomp_beam; k++) {
#pragma unroll 8
    for (int g = 0; g < d.ng; g++) acc += coef[g].de * p[k * d.comp_elems + (long long)g * 2 * d.lanes];
  }
  atomicAdd(flu + yz, (double)acc * scale);
}

template <typename st>
__device__ __forceinline__ st ldf(const st *p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <typename st, typename acc_t>
__device__ __forceinline__ void stf(st *p, acc_t v) { *p = (st)v; }
template <>
__device__ __forceinline__ void stf<__nv_bfloat16, float>(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// src[g][a][yz] = du dv sum_a' P2[g][a][a'] R[g][a'][yz]  (Remark 1): one GEMM
// of [na x na] by [na x nyz] per group, 64x64 output tiles, 16-deep k steps,
// 4x4 outputs per thread; acc is the accumulation type.
template <typename st, typename acc_t>
__global__ void __launch_bounds__(256) k_source_cc(const st *__restrict__ p2, const st *__restrict__ r, st *__restrict__ src,
                                                    int na, int nyz, int ng, long long gb0, acc_t dudv) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ acc_t As[BK][BM + 1];
  __shared__ acc_t Bs[BK][BN];
  const long long gb = gb0 + blockIdx.z;  // beam * ng + g
  const int g = (int)(gb % ng);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const st *A = p2 + (long long)g * na * na;
  const st *B = r + (long long)gb * na * nyz;
  st *C = src + (long long)gb * na * nyz;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  acc_t acc[4][4] = {};
  for (int k0 = 0; k0 < na; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      const int mm = e / BK, kk = e % BK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < na && gk < na) ? (acc_t)ldf(A + (long long)gm * na + gk) : acc_t(0);
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      const int kk = e / BN, nn = e % BN;
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < na && gn < nyz) ? (acc_t)ldf(B + (long long)gk * nyz + gn) : acc_t(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk++) {
      acc_t av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; i++) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; j++) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx + 16 * j;
      if (gm < na && gn < nyz) stf<st, acc_t>(C + (long long)gm * nyz + gn, acc[i][j] * dudv);
    }
}

// Energy-summed source input of one state (no trapezoid):
// R_g = T_g / dE_g,  T_g = rho q1_g psi^1_g + decay_g T_{g+1}  (Remark 1 with
// the exponential P^1), one thread per lane.
template <typename real, typename st>
__global__ void k_source_input(const real *__restrict__ psi, const real *__restrict__ rho_yz,
                               const GroupCoef<real> *__restrict__ coef, st *__restrict__ r, Dims d) {
  const long long lane = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (lane >= d.lanes) return;
  const real rho = rho_yz[lane % d.nyz];
  real t = 0;
  for (int g = d.ng - 1; g >= 0; g--) {
    const GroupCoef<real> k = coef[g];
    t = rho * k.q1 * psi[(long long)g * 2 * d.lanes + lane] + k.decay * t;
    stf<st, real>(r + (long long)g * d.lanes + lane, t * k.inv_de);
  }
}

}  // namespace

cudaError_t launch_source_input(const LaunchCtx &lc, const Dims &d, const void *psi_k, const void *rho_yz,
                                const void *coef, void *r_out, int precision) {
  const unsigned blocks = (unsigned)((d.lanes + 255) / 256);
  if (precision == 0)
    k_source_input<double, double><<<blocks, 256, 0, lc.stream>>>(
        (const double *)psi_k, (const double *)rho_yz, (const GroupCoef<double> *)coef, (double *)r_out, d);
  else if (precision == 1)
    k_source_input<float, float><<<blocks, 256, 0, lc.stream>>>(
        (const float *)psi_k, (const float *)rho_yz, (const GroupCoef<float> *)coef, (float *)r_out, d);
  else
    k_source_input<float, __nv_bfloat16><<<blocks, 256, 0, lc.stream>>>(
        (const float *)psi_k, (const float *)rho_yz, (const GroupCoef<float> *)coef, (__nv_bfloat16 *)r_out, d);
  ++*lc.launches;
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_init(const LaunchCtx &lc, const Dims &d, real *psi0, const double *fe, const double *fa,
                        const double *fy, const double *fz) {
  dim3 grid((unsigned)d.na, (unsigned)(2 * d.ng));
  const size_t smem = (size_t)(d.ny + d.nz) * sizeof(real);
  if (smem <= 48 * 1024)
    k_init_rows<real><<<grid, d.nz >= 256 ? 256 : 128, smem, lc.stream>>>(psi0, fe, fa, fy, fz, d);
  else
    k_init<real><<<grid, 256, 0, lc.stream>>>(psi0, fe, fa, fy, fz, d);
  ++*lc.launches;
  return cudaGetLastError();
}

template <typename real>
cudaError_t launch_fluence(const LaunchCtx &lc, const Dims &d, const real *psi, int ncomp_beam,
                           const GroupCoef<real> *coef, double *flu_yz, double scale) {
  dim3 grid((d.nyz + 127) / 128, d.na);
  k_fluence<real><<<grid, 128, 0, lc.stream>>>(psi, ncomp_beam, coef, flu_yz, d, scale);
  ++*lc.launches;
  return cudaGetLastError();
}

// grid.z is limited to 65535 (beam, group) blocks per launch: larger batches
// go in chunks.
template <typename st, typename acc_t>
cudaError_t launch_source_cc(const LaunchCtx &lc, const Dims &d, const st *p2, const st *r, st *src, acc_t dudv,
                             int nbatch) {
  const long long total = (long long)d.ng * nbatch;
  for (long long z0 = 0; z0 < total; z0 += 65535) {
    const long long cnt = total - z0 < 65535 ? total - z0 : 65535;
    dim3 grid((d.nyz + 63) / 64, (d.na + 63) / 64, (unsigned)cnt);
    k_source_cc<st, acc_t><<<grid, 256, 0, lc.stream>>>(p2, r, src, d.na, d.nyz, d.ng, z0, dudv);
    ++*lc.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// BF16 operands, FP32 accumulation on the CUDA cores (reference form of the
// tensor-core contraction).
cudaError_t launch_source_bf16_cc(const LaunchCtx &lc, const Dims &d, const __nv_bfloat16 *p2, const __nv_bfloat16 *r,
                                  __nv_bfloat16 *src, double dudv, int nbatch) {
  return launch_source_cc<__nv_bfloat16, float>(lc, d, p2, r, src, (float)dudv, nbatch);
}

cudaError_t launch_source_tc(const LaunchCtx &lc, const Dims &d, const __nv_bfloat16 *p2, const __nv_bfloat16 *r,
                             __nv_bfloat16 *src, double dudv, int nbatch);

template <typename real, typename st>
cudaError_t launch_source(const LaunchCtx &lc, const Dims &d, const st *p2, const st *r, st *src, double dudv,
                          int nbatch) {
  if constexpr (sizeof(st) == 2) {
    return launch_source_tc(lc, d, p2, r, src, dudv, nbatch);
  } else {
    return launch_source_cc<st, st>(lc, d, p2, r, src, (st)dudv, nbatch);
  }
}

template cudaError_t launch_init<double>(const LaunchCtx &, const Dims &, double *, const double *, const double *,
                                         const double *, const double *);
template cudaError_t launch_init<float>(const LaunchCtx &, const Dims &, float *, const double *, const double *,
                                        const double *, const double *);
template cudaError_t launch_fluence<double>(const LaunchCtx &, const Dims &, const double *, int,
                                            const GroupCoef<double> *, double *, double);
template cudaError_t launch_fluence<float>(const LaunchCtx &, const Dims &, const float *, int,
                                           const GroupCoef<float> *, double *, double);
template cudaError_t launch_source<double, double>(const LaunchCtx &, const Dims &, const double *, const double *,
                                                   double *, double, int);
template cudaError_t launch_source<float, float>(const LaunchCtx &, const Dims &, const float *, const float *, float *,
                                                 double, int);
template cudaError_t launch_source<float, __nv_bfloat16>(const LaunchCtx &, const Dims &, const __nv_bfloat16 *,
                                                         const __nv_bfloat16 *, __nv_bfloat16 *, double, int);

}  // namespace pbs
