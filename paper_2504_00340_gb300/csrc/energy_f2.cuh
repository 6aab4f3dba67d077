// energy_f2.cuh -- device code of the packed FP32 energy substep E(h)
// (Section 3.2 with T = 0, Crank-Nicolson; see k_energy_f2.cu for the
// design), shared by the per-substep kernels of k_energy_f2.cu and the
// persistent batch kernel of k_batch.cu.  Everything sits in an unnamed
// namespace: each translation unit that includes it gets its own copy.
#pragma once

#include "pbs_internal.cuh"

namespace pbs {
namespace {
namespace en {

constexpr int kX = 32;     // threads along the lateral axis (64 lateral points)
constexpr int kA = 2;      // angles per thread
constexpr int kU = 2;      // groups per prefetch block

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// c - a (via a * -1 + c)
__device__ __forceinline__ float2 rsub2(float2 a, float2 c) { return __ffma2_rn(a, make_float2(-1.f, -1.f), c); }

// Group constants duplicated into pairs (one 8-byte shared load per use).
struct GroupPair {
  float2 sm, sp, sig, ehat, dq, dq3, eh3, de, q1, decay, inv_de, pad;
};

template <typename st>
__device__ __forceinline__ float2 load_pair(const st *p);
template <>
__device__ __forceinline__ float2 load_pair<float>(const float *p) { return *reinterpret_cast<const float2 *>(p); }
template <>
__device__ __forceinline__ float2 load_pair<__nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
}
template <typename st>
__device__ __forceinline__ void store_pair(st *p, float2 v);
template <>
__device__ __forceinline__ void store_pair<float>(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
template <>
__device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16 *p, float2 v) {
  *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(v);
}

// Coefficients of one CN substep at (lateral pair, group), shared by angles.
struct Coef2 {
  float2 am, ap, ap3, a11, a22, p1, p2, p3, p4, c1n, c2, c3;
  __device__ __forceinline__ void make(const GroupPair &k, float2 rc) {
    am = mul2(rc, k.sm);
    ap = mul2(rc, k.sp);
    const float2 sg = mul2(rc, k.sig);
    const float2 u = add2(am, sg);              // m00 - 1
    const float2 m00 = add2(u, f2(1.f));
    const float2 m11 = add2(m00, add2(am, ap));  // 1 + ap + 2 am + sg
    ap3 = mul2(ap, f2(3.f));
    const float2 det = fma2(am, ap3, mul2(m00, m11));
    const float2 inv = make_float2(__fdividef(1.f, det.x), __fdividef(1.f, det.y));
    a11 = rsub2(u, f2(1.f));
    a22 = rsub2(m11, f2(2.f));
    p1 = mul2(m11, inv);
    p2 = mul2(am, inv);
    p3 = mul2(m00, inv);
    p4 = mul2(mul2(ap3, f2(-1.f)), inv);
    // deposited energy t = -c1n y1 + c2 y2 + c3 carry (+ c ehat s)
    c1n = fma2(k.ehat, u, mul2(k.dq, ap3));
    c2 = rsub2(mul2(k.dq, add2(u, add2(am, ap))), mul2(k.ehat, am));
    c3 = mul2(k.eh3, ap);
  }
};

// One angle through one substep: old (o1, o2) -> new (x1, x2); s = source.
template <bool HAS_SRC>
__device__ __forceinline__ void step_angle(const Coef2 &q, float2 cs, float2 o1, float2 o2, float2 s, float2 &carry,
                                           float2 &x1, float2 &x2, float2 &y1, float2 &Y1, float2 &Y2, float2 &CY) {
  float2 r0 = fma2(q.a11, o1, fma2(q.am, o2, mul2(q.ap, carry)));
  if (HAS_SRC) r0 = fma2(cs, s, r0);
  const float2 r1 = fma2(q.ap3, rsub2(o1, carry), mul2(q.a22, o2));
  x1 = fma2(q.p1, r0, mul2(q.p2, r1));
  x2 = fma2(q.p3, r1, mul2(q.p4, r0));
  y1 = add2(o1, x1);
  const float2 y2 = add2(o2, x2);
  Y1 = add2(Y1, y1);
  Y2 = add2(Y2, y2);
  CY = add2(CY, carry);
  carry = rsub2(y2, y1);
}

// Hint the L2 to fetch a line that a later group of the scan will read.
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Groups ahead of the scan whose psi and source rows the pass asks the L2
// for: the per-group loads are small (8-byte psi and 4-byte BF16 source
// pairs per thread), so the register prefetch of kU groups alone leaves the
// warps waiting on DRAM latency (on the 180 MeV slab workload the
// source-reading pass ran at 48 % of HBM).  Measured: 8 groups cut the energy
// time of that march by 10 % and of the K = 3 random-density march by 22 %;
// 16 was slower than none; 5 is a little faster than 8.
constexpr int kPF = 5;

// TwoSum compensated accumulation s + x (branch-free).
__device__ __forceinline__ void two_sum(float2 &s, float2 &c, float2 x) {
  const float2 t = add2(s, x);
  const float2 bp = rsub2(s, t);                          // t - s
  const float2 e = add2(rsub2(rsub2(bp, t), s), rsub2(bp, x));  // (s - (t - bp)) + (x - bp)
  c = add2(c, e);
  s = t;
}

// One block of the pass: block (bx, by, bz) of the grid
// ((nyz/2 + kX-1)/kX, (na + kY kA-1)/(kY kA), beams), thread (tx, ty) of the
// kX x kY block; smem_raw holds the group table (sizeof(GroupPair) * ng).
template <typename st, bool HAS_SRC, bool HAS_R, bool TWO, int kY>
__device__ __forceinline__ void energy_f2_tile(int bx, int by, int bz, int tx, int ty, unsigned char *smem_raw,
                                               Dims d, float *__restrict__ psi, const st *__restrict__ src_a,
                                               const st *__restrict__ src_b, st *__restrict__ r_a,
                                               st *__restrict__ r_b, const float *__restrict__ rho_a,
                                               const float *__restrict__ rho_b,
                                               const GroupCoef<float> *__restrict__ coef, double *__restrict__ dose_a,
                                               double *__restrict__ dose_b, double *__restrict__ flu, float c_a,
                                               float c_b, double dose_scale, double flu_scale, BeamStrides bs) {
  {
    const long long b = bz;
    psi += b * bs.psi;
    if (HAS_SRC) {
      src_a += b * bs.src;
      if (TWO) src_b += b * bs.src;
    }
    if (HAS_R) {
      r_a += b * bs.src;
      if (TWO) r_b += b * bs.src;
    }
    if (dose_a) dose_a += b * bs.dose;
    if (TWO && dose_b) dose_b += b * bs.dose;
    if (flu) flu += b * bs.flu;
  }
  GroupPair *tab = reinterpret_cast<GroupPair *>(smem_raw);
  const int tid = ty * kX + tx;
  for (int g = tid; g < d.ng; g += kX * kY) {
    const GroupCoef<float> k = coef[g];
    GroupPair &p = tab[g];
    p.sm = f2(k.sm);
    p.sp = f2(k.sp);
    p.sig = f2(k.sig);
    p.ehat = f2(k.ehat);
    p.dq = f2(k.dq);
    p.dq3 = f2(3.f * k.dq);
    p.eh3 = f2(k.ehat + 3.f * k.dq);
    p.de = f2(k.de);
    p.q1 = f2(k.q1);
    p.decay = f2(k.decay);
    p.inv_de = f2(k.inv_de);
    p.pad = f2(0.f);
  }
  __shared__ double red[3][kY][2 * kX];
  __syncthreads();

  const int yz = (bx * kX + tx) * 2;  // first of the thread's two lateral points
  const int a0 = (by * kY + ty) * kA;
  const bool lat_on = yz < d.nyz;
  bool on[kA];
#pragma unroll
  for (int j = 0; j < kA; j++) on[j] = lat_on && (a0 + j < d.na);
  const float2 rho2a = lat_on ? *reinterpret_cast<const float2 *>(rho_a + yz) : f2(0.f);
  const float2 rho2b = (TWO && lat_on) ? *reinterpret_cast<const float2 *>(rho_b + yz) : f2(0.f);
  const float2 rca = mul2(rho2a, f2(c_a)), rcb = mul2(rho2b, f2(c_b));
  const float2 csa = f2(c_a), csb = f2(c_b);
  const long long gstride = 2 * d.lanes;

  float *base[kA];
  const st *sa[kA];
  const st *sb[kA];
  st *ra[kA];
  st *rb[kA];
#pragma unroll
  for (int j = 0; j < kA; j++) {
    const long long lane = (long long)(a0 + j) * d.nyz + yz;
    base[j] = psi + lane;
    sa[j] = HAS_SRC ? src_a + lane : nullptr;
    sb[j] = (HAS_SRC && TWO) ? src_b + lane : nullptr;
    ra[j] = HAS_R ? r_a + lane : nullptr;
    rb[j] = (HAS_R && TWO) ? r_b + lane : nullptr;
  }

  float2 carA[kA], carB[kA], tsA[kA], tsB[kA];
#pragma unroll
  for (int j = 0; j < kA; j++) carA[j] = carB[j] = tsA[j] = tsB[j] = f2(0.f);
  float2 depA = f2(0.f), depAc = f2(0.f), depB = f2(0.f), depBc = f2(0.f), cnt = f2(0.f);

  float2 c1[kU][kA], c2_[kU][kA], cs_a[kU][kA], cs_b[kU][kA];
  float2 n1[kU][kA], n2[kU][kA], ns_a[kU][kA], ns_b[kU][kA];
  const int G = d.ng;
  auto fetch = [&](int g, float2 (&o1)[kA], float2 (&o2)[kA], float2 (&s_a)[kA], float2 (&s_b)[kA]) {
#pragma unroll
    for (int j = 0; j < kA; j++) {
      o1[j] = o2[j] = s_a[j] = s_b[j] = f2(0.f);
      if (on[j] && g >= 0) {
        o1[j] = *reinterpret_cast<const float2 *>(base[j] + g * gstride);
        o2[j] = *reinterpret_cast<const float2 *>(base[j] + g * gstride + d.lanes);
        if (HAS_SRC) s_a[j] = load_pair<st>(sa[j] + (long long)g * d.lanes);
        if (HAS_SRC && TWO) s_b[j] = load_pair<st>(sb[j] + (long long)g * d.lanes);
      }
    }
  };
#pragma unroll
  for (int u = 0; u < kU; u++) fetch(G - 1 - u, c1[u], c2_[u], cs_a[u], cs_b[u]);

  for (int gb = G - 1; gb >= 0; gb -= kU) {
    // L2 hints kPF groups ahead of the register prefetch
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const int g = gb - kPF - u;
      if (g >= 0) {
#pragma unroll
        for (int j = 0; j < kA; j++) {
          if (!on[j]) continue;
          prefetch_l2(base[j] + g * gstride);
          prefetch_l2(base[j] + g * gstride + d.lanes);
          if (HAS_SRC) prefetch_l2(sa[j] + (long long)g * d.lanes);
          if (HAS_SRC && TWO) prefetch_l2(sb[j] + (long long)g * d.lanes);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; u++) fetch(gb - kU - u, n1[u], n2[u], ns_a[u], ns_b[u]);
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const int g = gb - u;
      if (g < 0) break;
      const GroupPair k = tab[g];
      Coef2 qa;
      qa.make(k, rca);
      const float2 rqa = mul2(rho2a, k.q1);
      float2 Y1 = f2(0.f), Y2 = f2(0.f), CY = f2(0.f), X1 = f2(0.f), S = f2(0.f);
      float2 x1[kA], x2[kA];
#pragma unroll
      for (int j = 0; j < kA; j++) {
        float2 y1;
        step_angle<HAS_SRC>(qa, csa, c1[u][j], c2_[u][j], cs_a[u][j], carA[j], x1[j], x2[j], y1, Y1, Y2, CY);
        X1 = add2(X1, x1[j]);
        if (HAS_SRC) S = add2(S, cs_a[u][j]);
        if (HAS_R) {
          tsA[j] = fma2(rqa, y1, mul2(k.decay, tsA[j]));
          if (on[j]) store_pair<st>(ra[j] + (long long)g * d.lanes, mul2(tsA[j], k.inv_de));
        }
      }
      {
        float2 t = fma2(qa.c3, CY, rsub2(mul2(qa.c1n, Y1), mul2(qa.c2, Y2)));
        if (HAS_SRC) t = fma2(mul2(csa, k.ehat), S, t);
        two_sum(depA, depAc, mul2(t, f2(-1.f)));
        cnt = fma2(k.de, X1, cnt);
      }
      if (TWO) {
        Coef2 qb;
        qb.make(k, rcb);
        const float2 rqb = mul2(rho2b, k.q1);
        float2 Z1 = f2(0.f), Z2 = f2(0.f), CZ = f2(0.f), SB = f2(0.f);
#pragma unroll
        for (int j = 0; j < kA; j++) {
          float2 z1, z2, w1;
          step_angle<HAS_SRC>(qb, csb, x1[j], x2[j], cs_b[u][j], carB[j], z1, z2, w1, Z1, Z2, CZ);
          if (HAS_SRC) SB = add2(SB, cs_b[u][j]);
          if (HAS_R) {
            tsB[j] = fma2(rqb, w1, mul2(k.decay, tsB[j]));
            if (on[j]) store_pair<st>(rb[j] + (long long)g * d.lanes, mul2(tsB[j], k.inv_de));
          }
          x1[j] = z1;
          x2[j] = z2;
        }
        float2 t = fma2(qb.c3, CZ, rsub2(mul2(qb.c1n, Z1), mul2(qb.c2, Z2)));
        if (HAS_SRC) t = fma2(mul2(csb, k.ehat), SB, t);
        two_sum(depB, depBc, mul2(t, f2(-1.f)));
      }
#pragma unroll
      for (int j = 0; j < kA; j++) {
        if (on[j]) {
          *reinterpret_cast<float2 *>(base[j] + g * gstride) = x1[j];
          *reinterpret_cast<float2 *>(base[j] + g * gstride + d.lanes) = x2[j];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; u++)
#pragma unroll
      for (int j = 0; j < kA; j++) {
        c1[u][j] = n1[u][j];
        c2_[u][j] = n2[u][j];
        cs_a[u][j] = ns_a[u][j];
        cs_b[u][j] = ns_b[u][j];
      }
  }

  // reduce over the block's angle rows, add to the voxel tallies
  const bool any = on[0];
  const int xl = tx * 2;
  red[0][ty][xl] = any ? (double)depA.x + (double)depAc.x : 0.0;
  red[0][ty][xl + 1] = any ? (double)depA.y + (double)depAc.y : 0.0;
  red[1][ty][xl] = any ? (double)cnt.x : 0.0;
  red[1][ty][xl + 1] = any ? (double)cnt.y : 0.0;
  red[2][ty][xl] = (any && TWO) ? (double)depB.x + (double)depBc.x : 0.0;
  red[2][ty][xl + 1] = (any && TWO) ? (double)depB.y + (double)depBc.y : 0.0;
  __syncthreads();
  if (ty == 0 && lat_on) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
      double s_a = 0.0, s_f = 0.0, s_b = 0.0;
#pragma unroll
      for (int r = 0; r < kY; r++) {
        s_a += red[0][r][xl + h];
        s_f += red[1][r][xl + h];
        s_b += red[2][r][xl + h];
      }
      const int p = yz + h;
      const double ra_ = (double)rho_a[p];
      if (dose_a && ra_ > 0.0) atomicAdd(dose_a + p, s_a * dose_scale / ra_);
      if (flu) atomicAdd(flu + p, s_f * flu_scale);
      if (TWO) {
        const double rb_ = (double)rho_b[p];
        if (dose_b && rb_ > 0.0) atomicAdd(dose_b + p, s_b * dose_scale / rb_);
      }
    }
  }
}

}  // namespace en
}  // namespace
}  // namespace pbs
