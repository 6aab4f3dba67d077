// k_energy.cu -- energy substep E(h): Crank-Nicolson step of the DG-P1
// energy operator (Section 3.2, Eq. 0041-d with T = 0; Section 3.3), one
// thread per lane (y, z, u, v), descending scan over the energy groups.
//
// Per lane the operator is block upper-bidiagonal: group g couples to the
// group above through the upwind face value psi^1_{g+1} - psi^2_{g+1}.  With
// c = h/2 the CN system (I - c A) x = (I + c A) psi + c (src_old + src_new) is
// solved from the top group down, x_{G+1} = 0:
//   M_g x_g = (I + c A_gg) psi_g + c A_up (psi_{g+1} + x_{g+1}) + c src_g.
// Reading (sign of the phi^2-tested lower-face flux): +3 S_- (psi^1 - psi^2).
//
// Fused into the same pass (no extra HBM traffic beyond their own outputs):
//  * dose: the energy content lost in this substep, in the stable operator
//    form -c phi^T A (psi_old + x) - c phi^T src with phi = (E_g dE, dE^2/6),
//    accumulated per lane with compensated (Neumaier) summation, reduced over
//    8 angles in shared memory and added to the FP64 dose voxel;
//  * fluence after the substep (particle count du dv sum dE psi^1);
//  * the energy-summed source input of the next component (Remark 1 with the
//    exponential P^1 of Appendix A.4):  R_g = T_g / dE_g,
//    T_g = w_g + exp(-lambda (E_{g+1} - E_g)) T_{g+1},
//    w_g = lambda / Z_g rho sigma_g dE_g (psi^1_old + psi^1_new)_g,
//    i.e. the trapezoid (old + new) of the source of the next component.
#include "pbs_internal.cuh"

namespace pbs {

namespace {

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
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

// Neumaier compensated accumulation.
template <typename real>
__device__ __forceinline__ void comp_add(real &s, real &c, real x) {
  real t = s + x;
  c += (fabs(s) >= fabs(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

constexpr int kLanesX = 32;   // lateral points per block (coalesced)
constexpr int kAnglesY = 8;   // angles per block (reduced for the dose)
constexpr int kUnroll = 4;    // groups per prefetch block

template <typename real, typename st, bool HAS_SRC, bool HAS_R>
__global__ void __launch_bounds__(kLanesX *kAnglesY) k_energy(Dims d, real *__restrict__ psi,
                                                            const st *__restrict__ src, st *__restrict__ rout,
                                                            const real *__restrict__ rho_yz,
                                                            const GroupCoef<real> *__restrict__ coef,
                                                            double *__restrict__ dose, double *__restrict__ flu,
                                                            real c, double dose_scale, double flu_scale) {
  extern __shared__ unsigned char smem_raw[];
  GroupCoef<real> *tab = reinterpret_cast<GroupCoef<real> *>(smem_raw);
  const int tid = threadIdx.y * kLanesX + threadIdx.x;
  for (int g = tid; g < d.ng; g += kLanesX * kAnglesY) tab[g] = coef[g];
  __shared__ double red_dep[kAnglesY][kLanesX];
  __shared__ double red_flu[kAnglesY][kLanesX];
  __syncthreads();

  const int yz = blockIdx.x * kLanesX + threadIdx.x;
  const int a = blockIdx.y * kAnglesY + threadIdx.y;
  const bool active = (yz < d.nyz) && (a < d.na);
  const long long lane = (long long)a * d.nyz + yz;
  const long long gstride = 2 * d.lanes;
  const real rho = active ? rho_yz[yz] : real(0);
  const real rc = rho * c;

  real carry = 0;             // (psi^1 - psi^2)_{g+1} of old + new
  real dep = 0, dep_c = 0;    // deposited energy content (compensated)
  real cnt = 0;               // particle count after the substep
  real tsum = 0;              // source recursion T_g

  real *base = psi + lane;
  const st *sbase = HAS_SRC ? src + lane : nullptr;
  st *rbase = HAS_R ? rout + lane : nullptr;

  real cur1[kUnroll], cur2[kUnroll], cs[kUnroll];
  real nx1[kUnroll], nx2[kUnroll], ns[kUnroll];
  const int G = d.ng;
#pragma unroll
  for (int j = 0; j < kUnroll; j++) {
    int g = G - 1 - j;
    cur1[j] = cur2[j] = cs[j] = 0;
    if (active && g >= 0) {
      cur1[j] = base[g * gstride];
      cur2[j] = base[g * gstride + d.lanes];
      if (HAS_SRC) cs[j] = load_src<real, st>(sbase + (long long)g * d.lanes);
    }
  }
  for (int gb = G - 1; gb >= 0; gb -= kUnroll) {
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
      int g = gb - kUnroll - j;
      nx1[j] = nx2[j] = ns[j] = 0;
      if (active && g >= 0) {
        nx1[j] = base[g * gstride];
        nx2[j] = base[g * gstride + d.lanes];
        if (HAS_SRC) ns[j] = load_src<real, st>(sbase + (long long)g * d.lanes);
      }
    }
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
      const int g = gb - j;
      if (g < 0) break;
      const GroupCoef<real> &k = tab[g];
      const real o1 = cur1[j], o2 = cur2[j];
      const real am = rc * k.sm, ap = rc * k.sp, sg = rc * k.sig;
      // rhs = (I + c A_gg) psi_g + c A_up (old + new)_{g+1} + c src
      real r0 = (real(1) - am - sg) * o1 + am * o2 + ap * carry;
      real r1 = real(-3) * ap * o1 + (real(1) - ap - real(2) * am - sg) * o2 + real(3) * ap * carry;
      if (HAS_SRC) r0 += c * cs[j];
      // M = I - c A_gg = [[1+am+sg, -am], [3ap, 1+ap+2am+sg]]
      const real m00 = real(1) + am + sg;
      const real m11 = real(1) + ap + real(2) * am + sg;
      const real inv = recip(m00 * m11 + real(3) * am * ap);
      const real x1 = (m11 * r0 + am * r1) * inv;
      const real x2 = (m00 * r1 - real(3) * ap * r0) * inv;
      if (active) {
        base[g * gstride] = x1;
        base[g * gstride + d.lanes] = x2;
      }
      // deposited energy content: -(phi_g^T c A_gg y_g + phi_g^T c A_up y_{g+1}) - c phi^T src
      const real y1 = o1 + x1, y2 = o2 + x2;
      real t = k.ehat * ((-am - sg) * y1 + am * y2) + k.dq * (real(-3) * ap * y1 + (-ap - real(2) * am - sg) * y2) +
               (k.ehat + real(3) * k.dq) * ap * carry;
      if (HAS_SRC) t += c * k.ehat * cs[j];
      comp_add(dep, dep_c, -t);
      carry = y1 - y2;
      cnt += k.de * x1;
      if (HAS_R) {
        tsum = rho * k.q1 * y1 + k.decay * tsum;
        if (active) store_st<st, real>(rbase + (long long)g * d.lanes, tsum * k.inv_de);
      }
    }
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
      cur1[j] = nx1[j];
      cur2[j] = nx2[j];
      cs[j] = ns[j];
    }
  }

  // reduce over the block's 8 angles and add to the voxel tallies
  red_dep[threadIdx.y][threadIdx.x] = active ? (double)dep + (double)dep_c : 0.0;
  red_flu[threadIdx.y][threadIdx.x] = active ? (double)cnt : 0.0;
  __syncthreads();
  if (threadIdx.y == 0 && yz < d.nyz) {
    double sd = 0.0, sf = 0.0;
#pragma unroll
    for (int j = 0; j < kAnglesY; j++) {
      sd += red_dep[j][threadIdx.x];
      sf += red_flu[j][threadIdx.x];
    }
    const double r = (double)rho_yz[yz];
    if (dose && r > 0.0) atomicAdd(dose + yz, sd * dose_scale / r);
    if (flu) atomicAdd(flu + yz, sf * flu_scale);
  }
}

}  // namespace

template <typename real, typename st>
cudaError_t launch_energy(const LaunchCtx &lc, const Dims &d, real *psi_k, const st *src, st *r_out,
                          const real *rho_yz, const GroupCoef<real> *coef, double *dose_yz, double *flu_yz,
                          real c_half, double dose_scale, double flu_scale) {
  dim3 block(kLanesX, kAnglesY);
  dim3 grid((d.nyz + kLanesX - 1) / kLanesX, (d.na + kAnglesY - 1) / kAnglesY);
  size_t smem = sizeof(GroupCoef<real>) * d.ng;
  auto go = [&](auto kern) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, block, smem, lc.stream>>>(d, psi_k, src, r_out, rho_yz, coef, dose_yz, flu_yz, c_half,
                                           dose_scale, flu_scale);
    ++*lc.launches;
    return cudaGetLastError();
  };
  if (src && r_out) return go(k_energy<real, st, true, true>);
  if (src) return go(k_energy<real, st, true, false>);
  if (r_out) return go(k_energy<real, st, false, true>);
  return go(k_energy<real, st, false, false>);
}

template cudaError_t launch_energy<double, double>(const LaunchCtx &, const Dims &, double *, const double *,
                                                   double *, const double *, const GroupCoef<double> *, double *,
                                                   double *, double, double, double);
template cudaError_t launch_energy<float, float>(const LaunchCtx &, const Dims &, float *, const float *, float *,
                                                 const float *, const GroupCoef<float> *, double *, double *,
                                                 float, double, double);
template cudaError_t launch_energy<float, __nv_bfloat16>(const LaunchCtx &, const Dims &, float *,
                                                         const __nv_bfloat16 *, __nv_bfloat16 *, const float *,
                                                         const GroupCoef<float> *, double *, double *, float,
                                                         double, double);

}  // namespace pbs
