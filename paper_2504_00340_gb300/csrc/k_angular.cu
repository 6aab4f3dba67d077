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
#include "pbs_internal.cuh"

#include <cmath>

namespace pbs {

namespace {

// lateral points per CTA: one 128-byte row of the tile per angle
template <typename real>
__host__ __device__ constexpr int tile_w() { return sizeof(real) == 8 ? 16 : 32; }

// Orthonormal DST-I matrices sqrt(2/(N+1)) sin(pi (m+1)(i+1)/(N+1)) for every
// size N <= 16, row-major [m][i], in the constant bank (they depend on N
// only).  Indexed with compile-time offsets, so the multiply-adds read them
// as constant operands.
__constant__ float c_dst_f[kMaxAngle + 1][kMaxAngle * kMaxAngle];
__constant__ double c_dst_d[kMaxAngle + 1][kMaxAngle * kMaxAngle];

template <typename real>
struct DstTab;
template <>
struct DstTab<float> {
  template <int N>
  static __device__ __forceinline__ float at(int idx) { return c_dst_f[N][idx]; }
};
template <>
struct DstTab<double> {
  template <int N>
  static __device__ __forceinline__ double at(int idx) { return c_dst_d[N][idx]; }
};

template <typename real>
struct AngTables {
  real lam[kMaxAngle * kMaxAngle];  // eigenvalues [n][m]
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

__device__ __forceinline__ double mode_factor(double den) { return 2.0 / den - 1.0; }
__device__ __forceinline__ float mode_factor(float den) { return __fdividef(2.0f, den) - 1.0f; }

template <typename real, int NU, int NV>
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
    for (int n = 0; n < NV; n++) {
      // (1 + q lam) / (1 - q lam) = -1 + 2 / (1 - q lam); lam <= 0, so 1 - q lam >= 1
      const real den = real(1) - q * tb.lam[n * NU + t];
      y[n] *= mode_factor(den);
    }
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

template <typename real>
void fill_tables(AngTables<real> &tb, int nu, int nv, double du, double dv) {
  const double pi = 3.14159265358979323846;
  for (int n = 0; n < nv; n++)
    for (int m = 0; m < nu; m++)
      tb.lam[n * nu + m] = (real)((2.0 * std::cos(pi * (m + 1) / (nu + 1)) - 2.0) / (du * du) +
                                  (2.0 * std::cos(pi * (n + 1) / (nv + 1)) - 2.0) / (dv * dv));
}

template <typename real, int NU, int NV>
cudaError_t go(const LaunchCtx &lc, const Dims &d, real *psi, const real *rho_yz, const real *ts, double h, double du,
               double dv) {
  AngTables<real> tb;
  fill_tables(tb, NU, NV, du, dv);
  constexpr int NT = NU > NV ? NU : NV;
  constexpr int kTW = tile_w<real>();
  dim3 block(kTW, NT);
  // grid.y is limited to 65535 slab stacks per launch: larger batches go in chunks
  const long long total = (long long)d.ncomp * d.ng * 2;
  for (long long k0 = 0; k0 < total; k0 += 65535) {
    const long long cnt = total - k0 < 65535 ? total - k0 : 65535;
    dim3 grid((d.nyz + kTW - 1) / kTW, (unsigned)cnt);
    k_angular<real, NU, NV><<<grid, block, 0, lc.stream>>>(psi, rho_yz, ts, d.nyz, d.ng, (real)(0.25 * h), k0, tb);
    ++*lc.launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

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
  static float hf[kMaxAngle + 1][kMaxAngle * kMaxAngle];
  static double hd[kMaxAngle + 1][kMaxAngle * kMaxAngle];
  const double pi = 3.14159265358979323846;
  for (int n = 1; n <= kMaxAngle; n++)
    for (int m = 0; m < n; m++)
      for (int i = 0; i < n; i++) {
        const double v = std::sqrt(2.0 / (n + 1)) * std::sin(pi * (m + 1) * (i + 1) / (n + 1));
        hd[n][m * n + i] = v;
        hf[n][m * n + i] = (float)v;
      }
  cudaError_t e = cudaMemcpyToSymbol(c_dst_f, hf, sizeof(hf));
  if (e != cudaSuccess) return e;
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
