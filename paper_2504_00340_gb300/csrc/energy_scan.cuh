// energy_scan.cuh -- per-lane pieces shared by the scalar energy kernels
// (k_energy.cu, k_energy_strag.cu): storage conversions, the Neumaier
// accumulator and the state of one Crank-Nicolson scan over the groups.
#pragma once

#include "pbs_internal.cuh"

namespace pbs {
namespace escan {

template <typename real, typename st>
__device__ __forceinline__ real load_src(const st *p) { return static_cast<real>(*p); }
template <>
__device__ __forceinline__ float load_src<float, __nv_bfloat16>(const __nv_bfloat16 *p) {
  return __bfloat162float(*p);
}

template <typename st, typename real>
__device__ __forceinline__ void store_st(st *p, real v) { *p = static_cast<st>(v); }
template <>
__device__ __forceinline__ void store_st<__nv_bfloat16, float>(__nv_bfloat16 *p, float v) {
  *p = __float2bfloat16_rn(v);
}

__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }  // ~1 ulp, ample for FP32 psi

// Neumaier compensated accumulation.
template <typename real>
__device__ __forceinline__ void comp_add(real &s, real &c, real x) {
  real t = s + x;
  c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// Per-lane state of one CN scan.
template <typename real>
struct Scan {
  real rho, rc, c;
  real carry;        // (psi^1 - psi^2)_{g+1} of old + new
  real dep, dep_c;   // deposited energy content (compensated)
  real tsum;         // source recursion T_g

  __device__ __forceinline__ void init(real rho_, real c_) {
    rho = rho_;
    c = c_;
    rc = rho_ * c_;
    carry = dep = dep_c = tsum = real(0);
  }
  // One group: old (o1, o2) -> new (x1, x2); s = src_old + src_new (or 0).
  // Returns y1 = o1 + x1 for the source recursion of the next component.
  template <bool HAS_SRC>
  __device__ __forceinline__ real group(const GroupCoef<real> &k, real o1, real o2, real s, real &x1, real &x2) {
    const real am = rc * k.sm, ap = rc * k.sp, sg = rc * k.sig;
    real r0 = (real(1) - am - sg) * o1 + am * o2 + ap * carry;
    const real r1 = real(-3) * ap * o1 + (real(1) - ap - real(2) * am - sg) * o2 + real(3) * ap * carry;
    if (HAS_SRC) r0 += c * s;
    // M = I - c A_gg = [[1+am+sg, -am], [3ap, 1+ap+2am+sg]]
    const real m00 = real(1) + am + sg;
    const real m11 = real(1) + ap + real(2) * am + sg;
    const real inv = recip(m00 * m11 + real(3) * am * ap);
    x1 = (m11 * r0 + am * r1) * inv;
    x2 = (m00 * r1 - real(3) * ap * r0) * inv;
    // deposited energy content: -(phi_g^T c A_gg y_g + phi_g^T c A_up y_{g+1}) - c phi^T src
    const real y1 = o1 + x1, y2 = o2 + x2;
    real t = k.ehat * ((-am - sg) * y1 + am * y2) + k.dq * (real(-3) * ap * y1 + (-ap - real(2) * am - sg) * y2) +
             (k.ehat + real(3) * k.dq) * ap * carry;
    if (HAS_SRC) t += c * k.ehat * s;
    comp_add(dep, dep_c, -t);
    carry = y1 - y2;
    return y1;
  }
  // The same group with an explicit term: (e0, e1) = St psi_old at g, the
  // straggling operator per unit density applied to the old state (times 2,
  // so that rho c (e0, e1) is its contribution over the substep).  It joins
  // the right-hand side and the deposited energy content.
  template <bool HAS_SRC>
  __device__ __forceinline__ real group_x(const GroupCoef<real> &k, real o1, real o2, real s, real e0, real e1,
                                          real &x1, real &x2) {
    const real am = rc * k.sm, ap = rc * k.sp, sg = rc * k.sig;
    real r0 = (real(1) - am - sg) * o1 + am * o2 + ap * carry + rc * e0;
    const real r1 = real(-3) * ap * o1 + (real(1) - ap - real(2) * am - sg) * o2 + real(3) * ap * carry + rc * e1;
    if (HAS_SRC) r0 += c * s;
    const real m00 = real(1) + am + sg;
    const real m11 = real(1) + ap + real(2) * am + sg;
    const real inv = recip(m00 * m11 + real(3) * am * ap);
    x1 = (m11 * r0 + am * r1) * inv;
    x2 = (m00 * r1 - real(3) * ap * r0) * inv;
    const real y1 = o1 + x1, y2 = o2 + x2;
    real t = k.ehat * ((-am - sg) * y1 + am * y2) + k.dq * (real(-3) * ap * y1 + (-ap - real(2) * am - sg) * y2) +
             (k.ehat + real(3) * k.dq) * ap * carry + rc * (k.ehat * e0 + k.dq * e1);
    if (HAS_SRC) t += c * k.ehat * s;
    comp_add(dep, dep_c, -t);
    carry = y1 - y2;
    return y1;
  }
};

}  // namespace escan
}  // namespace pbs
