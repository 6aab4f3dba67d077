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

// The same matrices hold only N/2 distinct magnitudes: with q = (m+1)(i+1)
// mod 2(N+1) and k = q mod (N+1), entry (m, i) is zero when k = 0, else
// sign * sqrt(2/(N+1)) sin(pi k'/(N+1)) with k' = min(k, N+1-k) <= N/2 and
// sign = -1 exactly when q > N+1.  c_dst_mag holds those magnitudes for each
// even N (k' = 1 .. N/2 at offset mag_off(N)).
__host__ __device__ constexpr int mag_off(int n) { return n <= 2 ? 0 : mag_off(n - 2) + (n - 2) / 2; }
constexpr int kMagEntries = mag_off(kMaxAngle + 2);
__constant__ float c_dst_mag[kMagEntries];
__host__ __device__ constexpr int dst_q(int n, int m, int i) { return ((m + 1) * (i + 1)) % (2 * (n + 1)); }
__host__ __device__ constexpr int dst_k(int n, int m, int i) {
  return dst_q(n, m, i) % (n + 1) <= n / 2 ? dst_q(n, m, i) % (n + 1) : (n + 1) - dst_q(n, m, i) % (n + 1);
}
__host__ __device__ constexpr bool dst_neg(int n, int m, int i) { return dst_q(n, m, i) > n + 1; }

// Fill this translation unit's c_dst_f2 and c_dst_mag (synchronous).
cudaError_t upload_dst_f2() {
  static float2 h[kDstEntries];
  static float hm[kMagEntries];
  const double pi = 3.14159265358979323846;
  for (int n = 2; n <= kMaxAngle; n += 2) {
    for (int k = 1; k <= n / 2; k++)
      hm[mag_off(n) + k - 1] = (float)(std::sqrt(2.0 / (n + 1)) * std::sin(pi * k / (n + 1)));
    // the pair table from the same FP32 magnitudes (exact zeros), so that both
    // forms of the transform compute the same values
    for (int m = 0; m < n; m++)
      for (int i = 0; i < n; i++) {
        const int k = dst_k(n, m, i);
        const float v = k == 0 ? 0.0f : (dst_neg(n, m, i) ? -hm[mag_off(n) + k - 1] : hm[mag_off(n) + k - 1]);
        h[dst_off(n) + m * n + i] = make_float2(v, v);
      }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_dst_f2, h, sizeof(h));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_dst_mag, hm, sizeof(hm));
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

// The N/2 magnitudes of size N as duplicated pairs in registers, read
// through an opaque move so that the compiler keeps them there: used as
// constant-bank operands, every packed multiply-add needs its own move of the
// pair into registers first.
template <int N>
struct DstMag {
  float2 v[N / 2];
  __device__ __forceinline__ void load() {
#pragma unroll
    for (int k = 0; k < N / 2; k++) {
      float a;
      asm volatile("mov.b32 %0, %1;" : "=f"(a) : "f"(c_dst_mag[mag_off(N) + k]));
      v[k] = make_float2(a, a);
    }
  }
};

// dst_apply2 with the coefficients from registers: the magnitude and sign of
// every entry are known at compile time (zero entries skipped).
template <int N>
__device__ __forceinline__ void dst_apply2r(const float2 (&x)[N], float2 (&y)[N], const DstMag<N> &c) {
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
    for (int m = 0; m < N; m++) {
      const int k = dst_k(N, m, i);
      if (k == 0) continue;
      const float2 w = c.v[k - 1];
      const float2 v = (m & 1) ? o[i] : e[i];
      y[m] = dst_neg(N, m, i) ? fma2(make_float2(-w.x, -w.y), v, y[m]) : fma2(w, v, y[m]);
    }
}

// The v-direction magnitudes: the u set itself when the sizes agree.
template <int A, int B>
__device__ __forceinline__ const DstMag<B> &mag_pick(const DstMag<A> &a, const DstMag<B> &b) {
  if constexpr (A == B)
    return a;
  else
    return b;
}

// The transform of size N from the constant-bank table, or (REGC) from the
// register magnitudes.
template <int N, bool REGC>
__device__ __forceinline__ void dst_apply2x(const float2 (&x)[N], float2 (&y)[N], const DstMag<N> &c) {
  if constexpr (REGC)
    dst_apply2r<N>(x, y, c);
  else
    dst_apply2<N>(x, y);
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
template <int NU, int NV, bool EXACT, bool REGC = false>
__device__ __forceinline__ void angular_f2_tile(float *__restrict__ psi, const float *__restrict__ rho_yz,
                                                const float *__restrict__ ts, int nyz, int ng, float hq,
                                                long long kgc, int bx, int x, int t, unsigned char *smem_raw,
                                                const AngTables<float> &tb) {
  constexpr int NA = NU * NV;
  DstMag<NU> cu;
  DstMag<NV> cv_own;  // loaded only when NV != NU (else the u set serves both)
  if constexpr (REGC) {
    cu.load();
    if constexpr (NU != NV) cv_own.load();
  }
  const DstMag<NV> &cv = mag_pick<NU, NV>(cu, cv_own);
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
    dst_apply2x<NU, REGC>(r, y, cu);
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
    dst_apply2x<NV, REGC>(c, y, cv);
#pragma unroll
    for (int n = 0; n < NV; n++) {
      const float l = tb.lam[n * NU + t];
      y[n] = scale_mode2<EXACT>(y[n], q, l);
    }
    dst_apply2x<NV, REGC>(y, c, cv);
#pragma unroll
    for (int j = 0; j < NV; j++) tile[j * NU + t][x] = c[j];
  }
  __syncthreads();
  if (t < NV) {
    float2 r[NU], y[NU];
#pragma unroll
    for (int i = 0; i < NU; i++) r[i] = tile[t * NU + i][x];
    dst_apply2x<NU, REGC>(r, y, cu);
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
template <int NU, int NV, bool EXACT, int R, bool REGC = false>
__device__ __forceinline__ void angular_f2_tiles(float *__restrict__ psi, const float *__restrict__ rho_yz,
                                                 const float *__restrict__ ts, int nyz, int ng, float hq,
                                                 long long kgc0, long long kstride, long long nkgc, int bx, int x,
                                                 int t, unsigned char *smem_raw, const AngTables<float> &tb) {
  constexpr int NA = NU * NV;
  DstMag<NU> cu;
  DstMag<NV> cv_own;
  if constexpr (REGC) {
    cu.load();
    if constexpr (NU != NV) cv_own.load();
  }
  const DstMag<NV> &cv = mag_pick<NU, NV>(cu, cv_own);
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
      dst_apply2x<NU, REGC>(rr[r], y, cu);
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
      dst_apply2x<NV, REGC>(c, y, cv);
#pragma unroll
      for (int n = 0; n < NV; n++) {
        const float l = tb.lam[n * NU + t];
        y[n] = scale_mode2<EXACT>(y[n], q, l);
      }
      dst_apply2x<NV, REGC>(y, c, cv);
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
      dst_apply2x<NU, REGC>(rr, y, cu);
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
