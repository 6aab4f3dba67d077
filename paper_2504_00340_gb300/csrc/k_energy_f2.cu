// k_energy_f2.cu -- FP32 energy substep E(h), packed form.
//
// Same arithmetic as k_energy.cu (Crank-Nicolson step of the DG-P1 energy
// operator, Section 3.2 with T = 0; descending scan over the groups; fused
// dose, fluence and source input), reorganised for the FP32x2 datapath of
// sm_103a:
//  * a thread owns two adjacent lateral points (one float2 per load, 8-byte
//    coalesced) and A angles at those points;
//  * everything that depends on (lateral point, group) only -- the 2x2 CN
//    matrix, its inverse, the dose row vector -- is formed once per group
//    and shared by the thread's A angles, instead of once per angle;
//  * the per-angle recurrences run on float2 pairs with the packed
//    fma/mul/add instructions (two lateral points per instruction);
//  * the deposited energy of a group is formed from the angle sums of
//    y1 = psi^1_old + psi^1_new, y2 and the upwind carry (the dose row
//    vector does not depend on the angle), then accumulated per lateral
//    point with the branch-free TwoSum compensation.
// Used for FP32 psi when nyz is even and the group table fits in shared
// memory; other cases take k_energy.
#include "pbs_internal.cuh"
#include "energy_f2.cuh"

#include <type_traits>

namespace pbs {

namespace {

using namespace en;

template <typename st, bool HAS_SRC, bool HAS_R, bool TWO, int kY>
__global__ void __launch_bounds__(kX *kY, (HAS_SRC && HAS_R && TWO) ? 1 : 512 / (kX * kY))
    k_energy_f2(Dims d, float *__restrict__ psi, const st *__restrict__ src_a, const st *__restrict__ src_b,
                st *__restrict__ r_a, st *__restrict__ r_b, const float *__restrict__ rho_a,
                const float *__restrict__ rho_b, const GroupCoef<float> *__restrict__ coef,
                double *__restrict__ dose_a, double *__restrict__ dose_b, double *__restrict__ flu, float c_a,
                float c_b, double dose_scale, double flu_scale, BeamStrides bs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  energy_f2_tile<st, HAS_SRC, HAS_R, TWO, kY>(blockIdx.x, blockIdx.y, blockIdx.z, threadIdx.x, threadIdx.y, smem_raw, d,
                                             psi, src_a, src_b, r_a, r_b, rho_a, rho_b, coef, dose_a, dose_b, flu,
                                             c_a, c_b, dose_scale, flu_scale, bs);
}

// Straggling blocks of one group duplicated into pairs (three 16-byte
// broadcast loads: every thread of the block reads the same group).
__device__ __forceinline__ void load_strag(const StragCoef<float> *p, float2 (&v)[12]) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int i = 0; i < 3; i++) {
    const float4 t = __ldg(q + i);
    v[4 * i] = f2(t.x);
    v[4 * i + 1] = f2(t.y);
    v[4 * i + 2] = f2(t.z);
    v[4 * i + 3] = f2(t.w);
  }
}

// (e0, e1) = lo (l1, l2) + d (o1, o2) + up (u1, u2)
__device__ __forceinline__ void strag_apply(const float2 (&v)[12], float2 l1, float2 l2, float2 o1, float2 o2,
                                            float2 u1, float2 u2, float2 &e0, float2 &e1) {
  e0 = fma2(v[0], l1, fma2(v[1], l2, fma2(v[4], o1, fma2(v[5], o2, fma2(v[8], u1, mul2(v[9], u2))))));
  e1 = fma2(v[2], l1, fma2(v[3], l2, fma2(v[6], o1, fma2(v[7], o2, fma2(v[10], u1, mul2(v[11], u2))))));
}

// step_angle with the explicit straggling term rc (e0, e1) in the right-hand side.
template <bool HAS_SRC>
__device__ __forceinline__ void step_angle_x(const Coef2 &q, float2 cs, float2 rc, float2 o1, float2 o2, float2 s,
                                             float2 e0, float2 e1, float2 &carry, float2 &x1, float2 &x2,
                                             float2 &y1, float2 &Y1, float2 &Y2, float2 &CY) {
  float2 r0 = fma2(q.a11, o1, fma2(q.am, o2, fma2(q.ap, carry, mul2(rc, e0))));
  if (HAS_SRC) r0 = fma2(cs, s, r0);
  const float2 r1 = fma2(q.ap3, rsub2(o1, carry), fma2(q.a22, o2, mul2(rc, e1)));
  x1 = fma2(q.p1, r0, mul2(q.p2, r1));
  x2 = fma2(q.p3, r1, mul2(q.p4, r0));
  y1 = add2(o1, x1);
  const float2 y2 = add2(o2, x2);
  Y1 = add2(Y1, y1);
  Y2 = add2(Y2, y2);
  CY = add2(CY, carry);
  carry = rsub2(y2, y1);
}

// The same pass with energy straggling (explicit inside CN, as k_energy_strag
// in k_energy_strag.cu): each angle's right-hand side gains rho c St psi_old
// from psi_{g-1}, psi_g, psi_{g+1}, the deposited energy its phi-weighted
// angle sum; the fused pair's second scan runs one group behind the first.
template <typename st, bool HAS_SRC, bool HAS_R, bool TWO, int kY>
__global__ void __launch_bounds__(kX *kY, (TWO && (HAS_SRC || HAS_R)) ? 1 : 512 / (kX * kY))
    k_energy_f2_strag(Dims d, float *__restrict__ psi, const st *__restrict__ src_a, const st *__restrict__ src_b,
                st *__restrict__ r_a, st *__restrict__ r_b, const float *__restrict__ rho_a,
                const float *__restrict__ rho_b, const GroupCoef<float> *__restrict__ coef,
                const StragCoef<float> *__restrict__ strag, double *__restrict__ dose_a, double *__restrict__ dose_b, double *__restrict__ flu, float c_a,
                float c_b, double dose_scale, double flu_scale, BeamStrides bs) {
  {
    const long long b = blockIdx.z;
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
  GroupPair *tab = reinterpret_cast<GroupPair *>(smem_raw);
  const int tid = threadIdx.y * kX + threadIdx.x;
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

  const int yz = (blockIdx.x * kX + threadIdx.x) * 2;  // first of the thread's two lateral points
  const int a0 = (blockIdx.y * kY + threadIdx.y) * kA;
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
  // old psi at g + 1 per angle; for the second scan (one group behind): the
  // first scan's results at g + 1 and g + 2 and the second source at g + 1
  float2 op1[kA], op2[kA], mc1[kA], mc2[kA], mu1[kA], mu2[kA], sbc[kA];
#pragma unroll
  for (int j = 0; j < kA; j++) {
    carA[j] = carB[j] = tsA[j] = tsB[j] = f2(0.f);
    op1[j] = op2[j] = mc1[j] = mc2[j] = mu1[j] = mu2[j] = sbc[j] = f2(0.f);
  }
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

  // second scan at group gq; (l1, l2) = first scan's result at gq - 1
  auto second = [&](int gq, const float2 (&l1)[kA], const float2 (&l2)[kA]) {
    const GroupPair k = tab[gq];
    float2 sv[12];
    load_strag(strag + gq, sv);
    Coef2 qb;
    qb.make(k, rcb);
    const float2 rqb = mul2(rho2b, k.q1);
    float2 Z1 = f2(0.f), Z2 = f2(0.f), CZ = f2(0.f), SB = f2(0.f), E0 = f2(0.f), E1 = f2(0.f);
#pragma unroll
    for (int j = 0; j < kA; j++) {
      float2 e0, e1, z1, z2, w1;
      strag_apply(sv, l1[j], l2[j], mc1[j], mc2[j], mu1[j], mu2[j], e0, e1);
      E0 = add2(E0, e0);
      E1 = add2(E1, e1);
      step_angle_x<HAS_SRC>(qb, csb, rcb, mc1[j], mc2[j], sbc[j], e0, e1, carB[j], z1, z2, w1, Z1, Z2, CZ);
      if (HAS_SRC) SB = add2(SB, sbc[j]);
      if (HAS_R) {
        tsB[j] = fma2(rqb, w1, mul2(k.decay, tsB[j]));
        if (on[j]) store_pair<st>(rb[j] + (long long)gq * d.lanes, mul2(tsB[j], k.inv_de));
      }
      if (on[j]) {
        *reinterpret_cast<float2 *>(base[j] + gq * gstride) = z1;
        *reinterpret_cast<float2 *>(base[j] + gq * gstride + d.lanes) = z2;
      }
    }
    float2 t = fma2(qb.c3, CZ, rsub2(mul2(qb.c1n, Z1), mul2(qb.c2, Z2)));
    if (HAS_SRC) t = fma2(mul2(csb, k.ehat), SB, t);
    t = fma2(mul2(rcb, k.ehat), E0, fma2(mul2(rcb, k.dq), E1, t));
    two_sum(depB, depBc, mul2(t, f2(-1.f)));
  };

  for (int gb = G - 1; gb >= 0; gb -= kU) {
#pragma unroll
    for (int u = 0; u < kU; u++) fetch(gb - kU - u, n1[u], n2[u], ns_a[u], ns_b[u]);
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const int g = gb - u;
      if (g < 0) break;
      const GroupPair k = tab[g];
      float2 sv[12];
      load_strag(strag + g, sv);
      Coef2 qa;
      qa.make(k, rca);
      const float2 rqa = mul2(rho2a, k.q1);
      float2 Y1 = f2(0.f), Y2 = f2(0.f), CY = f2(0.f), X1 = f2(0.f), S = f2(0.f), E0 = f2(0.f), E1 = f2(0.f);
      float2 x1[kA], x2[kA];
#pragma unroll
      for (int j = 0; j < kA; j++) {
        // old psi at g - 1: the next register of this block, or the first of the next block (0 below g = 0)
        const float2 l1 = (u + 1 < kU) ? c1[u + 1][j] : n1[0][j];
        const float2 l2 = (u + 1 < kU) ? c2_[u + 1][j] : n2[0][j];
        float2 y1, e0, e1;
        strag_apply(sv, l1, l2, c1[u][j], c2_[u][j], op1[j], op2[j], e0, e1);
        E0 = add2(E0, e0);
        E1 = add2(E1, e1);
        step_angle_x<HAS_SRC>(qa, csa, rca, c1[u][j], c2_[u][j], cs_a[u][j], e0, e1, carA[j], x1[j], x2[j], y1, Y1,
                              Y2, CY);
        op1[j] = c1[u][j];
        op2[j] = c2_[u][j];
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
        t = fma2(mul2(rca, k.ehat), E0, fma2(mul2(rca, k.dq), E1, t));
        two_sum(depA, depAc, mul2(t, f2(-1.f)));
        cnt = fma2(k.de, X1, cnt);
      }
      if (TWO) {
        if (g + 1 < G) second(g + 1, x1, x2);
#pragma unroll
        for (int j = 0; j < kA; j++) {
          mu1[j] = mc1[j];
          mu2[j] = mc2[j];
          mc1[j] = x1[j];
          mc2[j] = x2[j];
          sbc[j] = cs_b[u][j];
        }
      } else {
#pragma unroll
        for (int j = 0; j < kA; j++) {
          if (on[j]) {
            *reinterpret_cast<float2 *>(base[j] + g * gstride) = x1[j];
            *reinterpret_cast<float2 *>(base[j] + g * gstride + d.lanes) = x2[j];
          }
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
  if (TWO && G > 0) {
    const float2 zero[kA] = {};
    second(0, zero, zero);
  }

  // reduce over the block's angle rows, add to the voxel tallies
  const bool any = on[0];
  const int xl = threadIdx.x * 2;
  red[0][threadIdx.y][xl] = any ? (double)depA.x + (double)depAc.x : 0.0;
  red[0][threadIdx.y][xl + 1] = any ? (double)depA.y + (double)depAc.y : 0.0;
  red[1][threadIdx.y][xl] = any ? (double)cnt.x : 0.0;
  red[1][threadIdx.y][xl + 1] = any ? (double)cnt.y : 0.0;
  red[2][threadIdx.y][xl] = (any && TWO) ? (double)depB.x + (double)depBc.x : 0.0;
  red[2][threadIdx.y][xl + 1] = (any && TWO) ? (double)depB.y + (double)depBc.y : 0.0;
  __syncthreads();
  if (threadIdx.y == 0 && lat_on) {
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

}  // namespace

bool energy_f2_supported(const Dims &d) {
  return (d.nyz % 2) == 0 && sizeof(GroupPair) * (size_t)d.ng <= 160 * 1024;
}

template <typename st>
cudaError_t launch_energy_f2(const LaunchCtx &lc, const Dims &d, float *psi_k, const EnergyHalf<float, st> &ha,
                             const EnergyHalf<float, st> *hb, const GroupCoef<float> *coef, double *flu_yz,
                             double dose_scale, double flu_scale, const BeamStrides &bs,
                             const StragCoef<float> *strag) {
  const int angles = lc.energy_angles;  // angles per block: kY rows x kA
  const size_t smem = sizeof(GroupPair) * d.ng;
  const bool has_src = ha.src != nullptr, has_r = ha.r_out != nullptr;
  const EnergyHalf<float, st> &b = hb ? *hb : ha;
  auto pick = [&](auto ky_tag) -> cudaError_t {
    constexpr int KY = decltype(ky_tag)::value;
    dim3 block(kX, KY);
    dim3 grid((d.nyz / 2 + kX - 1) / kX, (d.na + KY * kA - 1) / (KY * kA), d.nbeam);
    auto go = [&](auto kern) -> cudaError_t {
      if (smem + sizeof(double) * 3 * KY * 2 * kX > 48 * 1024) {  // dynamic table + static reduction buffer
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      kern<<<grid, block, smem, lc.stream>>>(d, psi_k, ha.src, b.src, ha.r_out, b.r_out, ha.rho, b.rho, coef,
                                             ha.dose, b.dose, flu_yz, ha.c, b.c, dose_scale, flu_scale, bs);
      ++*lc.launches;
      return cudaGetLastError();
    };
    auto go_s = [&](auto kern) -> cudaError_t {
      if (smem + sizeof(double) * 3 * KY * 2 * kX > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
      }
      kern<<<grid, block, smem, lc.stream>>>(d, psi_k, ha.src, b.src, ha.r_out, b.r_out, ha.rho, b.rho, coef, strag,
                                             ha.dose, b.dose, flu_yz, ha.c, b.c, dose_scale, flu_scale, bs);
      ++*lc.launches;
      return cudaGetLastError();
    };
    if (strag) {
#define PBS_E2S(S, R, T) \
  if (has_src == S && has_r == R && (hb != nullptr) == T) return go_s(k_energy_f2_strag<st, S, R, T, KY>);
      PBS_E2S(true, true, true) PBS_E2S(true, false, true) PBS_E2S(false, true, true) PBS_E2S(false, false, true)
      PBS_E2S(true, true, false) PBS_E2S(true, false, false) PBS_E2S(false, true, false) PBS_E2S(false, false, false)
#undef PBS_E2S
      return cudaErrorInvalidValue;
    }
#define PBS_E2(S, R, T) \
  if (has_src == S && has_r == R && (hb != nullptr) == T) return go(k_energy_f2<st, S, R, T, KY>);
    PBS_E2(true, true, true) PBS_E2(true, false, true) PBS_E2(false, true, true) PBS_E2(false, false, true)
    PBS_E2(true, true, false) PBS_E2(true, false, false) PBS_E2(false, true, false) PBS_E2(false, false, false)
#undef PBS_E2
    return cudaErrorInvalidValue;
  };
  if (angles == 4) return pick(std::integral_constant<int, 2>{});
  if (angles == 8) return pick(std::integral_constant<int, 4>{});
  if (angles == 16) return pick(std::integral_constant<int, 8>{});
  return cudaErrorInvalidConfiguration;
}

template cudaError_t launch_energy_f2<float>(const LaunchCtx &, const Dims &, float *, const EnergyHalf<float, float> &,
                                             const EnergyHalf<float, float> *, const GroupCoef<float> *, double *,
                                             double, double, const BeamStrides &, const StragCoef<float> *);
template cudaError_t launch_energy_f2<__nv_bfloat16>(const LaunchCtx &, const Dims &, float *,
                                                     const EnergyHalf<float, __nv_bfloat16> &,
                                                     const EnergyHalf<float, __nv_bfloat16> *,
                                                     const GroupCoef<float> *, double *, double, double,
                                                     const BeamStrides &, const StragCoef<float> *);

}  // namespace pbs
