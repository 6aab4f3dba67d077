// angular_f2.cuh -- device code of the packed FP32 angular substep A(h)
// (Section 3.4, Eqs. sd and fly; see k_angular.cu for the design), shared by
// the per-substep kernel of k_angular.cu and the persistent batch kernel of
// k_batch.cu.  Everything sits in an unnamed namespace: each translation unit
// that includes it gets its own copy, including the constant-bank sine table
// c_dst_f2, which each unit fills with its own upload_dst_f2().
#pragma once

#include <cmath>

#include "pbs_internal.cuh"

namespace pbs {
namespace {
namespace ang {

// Orthonormal DST-I matrices sqrt(2/(N+1)) sin(pi (m+1)(i+1)/(N+1)) for every
// even size N <= 16, row-major [m][i], one after another (size N at offset
// dst_off(N)); each FP32 entry twice, as the pair operand of the packed
// FP32x2 multiply-adds.
__host__ __device__ constexpr int dst_off(int n) { return n <= 2 ? 0 : dst_off(n - 2) + (n - 2) * (n - 2); }
constexpr int kDstEntries = dst_off(kMaxAngle + 2);
__constant__ float2 c_dst_f2[kDstEntries];

// Fill this translation unit's c_dst_f2 (synchronous).
cudaError_t upload_dst_f2() {
  static float2 h[kDstEntries];
  const double pi = 3.14159265358979323846;
  for (int n = 2; n <= kMaxAngle; n += 2)
    for (int m = 0; m < n; m++)
      for (int i = 0; i < n; i++) {
        const float v = (float)(std::sqrt(2.0 / (n + 1)) * std::sin(pi * (m + 1) * (i + 1) / (n + 1)));
        h[dst_off(n) + m * n + i] = make_float2(v, v);
      }
  return cudaMemcpyToSymbol(c_dst_f2, h, sizeof(h));
}

template <typename real>
struct AngTables {
  real lam[kMaxAngle * kMaxAngle];  // eigenvalues [n][m]
};

// Eigenvalues of the five-point Laplacian with zero Dirichlet values (Eq.
// fly): lam[n][m] = (2cos(pi (m+1)/(nu+1)) - 2)/du^2 + (2cos(pi (n+1)/(nv+1)) - 2)/dv^2.
template <typename real>
void fill_tables(AngTables<real> &tb, int nu, int nv, double du, double dv) {
  const double pi = 3.14159265358979323846;
  for (int n = 0; n < nv; n++)
    for (int m = 0; m < nu; m++)
      tb.lam[n * nu + m] = (real)((2.0 * std::cos(pi * (m + 1) / (nu + 1)) - 2.0) / (du * du) +
                                  (2.0 * std::cos(pi * (n + 1) / (nv + 1)) - 2.0) / (dv * dv));
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ double mode_factor(double den) { return 2.0 / den - 1.0; }
__device__ __forceinline__ float mode_factor(float den) { return __fdividef(2.0f, den) - 1.0f; }

// Factor of one sine mode over the step, ql = (h kappa / 4) lam <= 0:
// Crank-Nicolson (1 + ql) / (1 - ql) = -1 + 2 / (1 - ql), or the exact
// solution exp(2 ql) of the mode's ODE.
template <bool EXACT>
__device__ __forceinline__ double mode_scale(double ql) {
  return EXACT ? exp(2.0 * ql) : mode_factor(1.0 - ql);
}
template <bool EXACT>
__device__ __forceinline__ float mode_scale(float ql) {
  return EXACT ? expf(2.0f * ql) : mode_factor(1.0f - ql);
}

// y *= the mode's factor at two lateral points (q = h kappa / 4 of each, l
// the mode's eigenvalue).  Crank-Nicolson on FP32x2 pairs: den = 1 - q l
// (one packed FMA), the two reciprocals, 2 / den - 1 (one packed FMA), one
// packed multiply; the exact exponential per point.
template <bool EXACT>
__device__ __forceinline__ float2 scale_mode2(float2 y, float2 q, float l) {
  if constexpr (EXACT) {
    y.x *= mode_scale<true>(q.x * l);
    y.y *= mode_scale<true>(q.y * l);
    return y;
  } else {
    const float2 den = fma2(q, make_float2(-l, -l), make_float2(1.f, 1.f));
    float2 r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(den.y));
    return __fmul2_rn(y, fma2(make_float2(2.f, 2.f), r, make_float2(-1.f, -1.f)));
  }
}

// dst_apply on pairs (two lateral points per register pair).
template <int N>
__device__ __forceinline__ void dst_apply2(const float2 (&x)[N], float2 (&y)[N]) {
  constexpr int H = N / 2;
  float2 e[H], o[H];
#pragma unroll
  for (int i = 0; i < H; i++) {
    e[i] = add2(x[i], x[N - 1 - i]);
    o[i] = fma2(x[N - 1 - i], make_float2(-1.f, -1.f), x[i]);
  }
#pragma unroll
  for (int m = 0; m < N; m++) y[m] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < H; i++)
#pragma unroll
    for (int m = 0; m < N; m++) y[m] = fma2(c_dst_f2[dst_off(N) + m * N + i], (m & 1) ? o[i] : e[i], y[m]);
}

// As k_angular with each thread on two adjacent lateral points (one 8-byte
// load per row) and the transforms on FP32x2 pairs; kF2X threads (2 kF2X
// lateral points) per slab row, so that a warp covers two rows of 128 bytes
// and several CTAs fit an SM (one CTA's loads overlap another's transforms).
// nyz must be even.
constexpr int kF2X = 16;
// Slab stack kgc = (k * ng + g) * 2 + c, lateral block bx (2 kF2X points);
// thread (x, t) of the kF2X x max(NU, NV) block; smem_raw holds the
// transformed tile (NU NV kF2X float2).
template <int NU, int NV, bool EXACT>
__device__ __forceinline__ void angular_f2_tile(float *__restrict__ psi, const float *__restrict__ rho_yz,
                                                const float *__restrict__ ts, int nyz, int ng, float hq,
                                                long long kgc, int bx, int x, int t, unsigned char *smem_raw,
                                                const AngTables<float> &tb) {
  constexpr int NA = NU * NV;
  float2(*tile)[kF2X] = reinterpret_cast<float2(*)[kF2X]>(smem_raw);
  const int g = (int)((kgc / 2) % ng);
  const int yz = (bx * kF2X + x) * 2;
  const bool active = yz < nyz;
  float *base = psi + kgc * (long long)NA * nyz + yz;
  if (t < NV) {
    float2 r[NU], y[NU];
#pragma unroll
    for (int i = 0; i < NU; i++)
      r[i] = active ? *reinterpret_cast<const float2 *>(base + (long long)(t * NU + i) * nyz) : make_float2(0.f, 0.f);
    dst_apply2<NU>(r, y);
#pragma unroll
    for (int i = 0; i < NU; i++) tile[t * NU + i][x] = y[i];
  }
  __syncthreads();
  if (t < NU) {
    float2 q = make_float2(0.f, 0.f);
    if (active) {
      const float2 rr = *reinterpret_cast<const float2 *>(rho_yz + yz);
      const float w = hq * ts[g];
      q = make_float2(w * rr.x, w * rr.y);  // h kappa / 4
    }
    float2 c[NV], y[NV];
#pragma unroll
    for (int j = 0; j < NV; j++) c[j] = tile[j * NU + t][x];
    dst_apply2<NV>(c, y);
#pragma unroll
    for (int n = 0; n < NV; n++) {
      const float l = tb.lam[n * NU + t];
      y[n] = scale_mode2<EXACT>(y[n], q, l);
    }
    dst_apply2<NV>(y, c);
#pragma unroll
    for (int j = 0; j < NV; j++) tile[j * NU + t][x] = c[j];
  }
  __syncthreads();
  if (t < NV) {
    float2 r[NU], y[NU];
#pragma unroll
    for (int i = 0; i < NU; i++) r[i] = tile[t * NU + i][x];
    dst_apply2<NU>(r, y);
    if (active) {
#pragma unroll
      for (int i = 0; i < NU; i++) *reinterpret_cast<float2 *>(base + (long long)(t * NU + i) * nyz) = y[i];
    }
  }
}

// R slab stacks kgc0 + r * kstride (r < R; those >= nkgc are skipped) at one
// lateral block, each exactly as angular_f2_tile, interleaved phase by phase
// so that the loads of the R stacks are in flight together (latency hidden
// by independent work instead of by more resident warps).  smem_raw holds R
// tiles.
template <int NU, int NV, bool EXACT, int R>
__device__ __forceinline__ void angular_f2_tiles(float *__restrict__ psi, const float *__restrict__ rho_yz,
                                                 const float *__restrict__ ts, int nyz, int ng, float hq,
                                                 long long kgc0, long long kstride, long long nkgc, int bx, int x,
                                                 int t, unsigned char *smem_raw, const AngTables<float> &tb) {
  constexpr int NA = NU * NV;
  const int yz = (bx * kF2X + x) * 2;
  float *base[R];
  bool active[R];
  float2(*tile[R])[kF2X];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const long long kgc = kgc0 + r * kstride;
    active[r] = yz < nyz && kgc < nkgc;
    base[r] = psi + (active[r] ? kgc : 0) * (long long)NA * nyz + yz;
    tile[r] = reinterpret_cast<float2(*)[kF2X]>(smem_raw + (size_t)r * sizeof(float2) * NA * kF2X);
  }
  if (t < NV) {
    float2 rr[R][NU];
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
      for (int i = 0; i < NU; i++)
        rr[r][i] = active[r] ? *reinterpret_cast<const float2 *>(base[r] + (long long)(t * NU + i) * nyz)
                             : make_float2(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < R; r++) {
      float2 y[NU];
      dst_apply2<NU>(rr[r], y);
#pragma unroll
      for (int i = 0; i < NU; i++) tile[r][t * NU + i][x] = y[i];
    }
  }
  __syncthreads();
  if (t < NU) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      const long long kgc = kgc0 + r * kstride;
      const int g = (int)(((kgc < nkgc ? kgc : 0) / 2) % ng);
      float2 q = make_float2(0.f, 0.f);
      if (active[r]) {
        const float2 rh = *reinterpret_cast<const float2 *>(rho_yz + yz);
        const float w = hq * ts[g];
        q = make_float2(w * rh.x, w * rh.y);  // h kappa / 4
      }
      float2 c[NV], y[NV];
#pragma unroll
      for (int j = 0; j < NV; j++) c[j] = tile[r][j * NU + t][x];
      dst_apply2<NV>(c, y);
#pragma unroll
      for (int n = 0; n < NV; n++) {
        const float l = tb.lam[n * NU + t];
        y[n] = scale_mode2<EXACT>(y[n], q, l);
      }
      dst_apply2<NV>(y, c);
#pragma unroll
      for (int j = 0; j < NV; j++) tile[r][j * NU + t][x] = c[j];
    }
  }
  __syncthreads();
  if (t < NV) {
#pragma unroll
    for (int r = 0; r < R; r++) {
      float2 rr[NU], y[NU];
#pragma unroll
      for (int i = 0; i < NU; i++) rr[i] = tile[r][t * NU + i][x];
      dst_apply2<NU>(rr, y);
      if (active[r]) {
#pragma unroll
        for (int i = 0; i < NU; i++) *reinterpret_cast<float2 *>(base[r] + (long long)(t * NU + i) * nyz) = y[i];
      }
    }
  }
}

}  // namespace ang
}  // namespace
}  // namespace pbs
