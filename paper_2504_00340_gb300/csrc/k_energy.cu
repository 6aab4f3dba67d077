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
//
// Two consecutive E substeps (the closing E(h/2) of depth step s and the
// opening E(h/2) of step s+1, which Strang splitting puts back to back) are
// fused: both scans descend in g, so the second consumes the first's output
// group by group and psi makes one trip through HBM instead of two.
#include "energy_scan.cuh"

#include <type_traits>

namespace pbs {

namespace {

using namespace escan;

constexpr int kLanesX = 32;   // lateral points per block (coalesced)
constexpr int kUnroll = 4;    // groups per prefetch block
// Angles per block (reduced in shared memory for the dose): a tile-shape
// knob of the autotuner, 4, 8 (default) or 16.

template <typename real, typename st, bool HAS_SRC, bool HAS_R, bool TWO, int kAnglesY>
__global__ void __launch_bounds__(kLanesX *kAnglesY)
    k_energy(Dims d, real *__restrict__ psi, const st *__restrict__ src_a, const st *__restrict__ src_b,
             st *__restrict__ r_a, st *__restrict__ r_b, const real *__restrict__ rho_a,
             const real *__restrict__ rho_b, const GroupCoef<real> *__restrict__ coef, double *__restrict__ dose_a,
             double *__restrict__ dose_b, double *__restrict__ flu, real c_a, real c_b, double dose_scale,
             double flu_scale, BeamStrides bs) {
  // beam blockIdx.z: shift every per-beam pointer to its copy
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
  extern __shared__ unsigned char smem_raw[];
  GroupCoef<real> *tab = reinterpret_cast<GroupCoef<real> *>(smem_raw);
  const int tid = threadIdx.y * kLanesX + threadIdx.x;
  for (int g = tid; g < d.ng; g += kLanesX * kAnglesY) tab[g] = coef[g];
  __shared__ double red[3][kAnglesY][kLanesX];
  __syncthreads();

  const int yz = blockIdx.x * kLanesX + threadIdx.x;
  const int a = blockIdx.y * kAnglesY + threadIdx.y;
  const bool active = (yz < d.nyz) && (a < d.na);
  const long long lane = (long long)a * d.nyz + yz;
  const long long gstride = 2 * d.lanes;

  Scan<real> A, B;
  A.init(active ? rho_a[yz] : real(0), c_a);
  if (TWO) B.init(active ? rho_b[yz] : real(0), c_b);
  real cnt = 0;  // particle count after the first scan

  real *base = psi + lane;
  const st *sa = HAS_SRC ? src_a + lane : nullptr;
  const st *sb = (HAS_SRC && TWO) ? src_b + lane : nullptr;
  st *ra = HAS_R ? r_a + lane : nullptr;
  st *rb = (HAS_R && TWO) ? r_b + lane : nullptr;

  real cur1[kUnroll], cur2[kUnroll], csa[kUnroll], csb[kUnroll];
  real nx1[kUnroll], nx2[kUnroll], nsa[kUnroll], nsb[kUnroll];
  const int G = d.ng;
#pragma unroll
  for (int j = 0; j < kUnroll; j++) {
    const int g = G - 1 - j;
    cur1[j] = cur2[j] = csa[j] = csb[j] = 0;
    if (active && g >= 0) {
      cur1[j] = base[g * gstride];
      cur2[j] = base[g * gstride + d.lanes];
      if (HAS_SRC) csa[j] = load_src<real, st>(sa + (long long)g * d.lanes);
      if (HAS_SRC && TWO) csb[j] = load_src<real, st>(sb + (long long)g * d.lanes);
    }
  }
  for (int gb = G - 1; gb >= 0; gb -= kUnroll) {
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
      const int g = gb - kUnroll - j;
      nx1[j] = nx2[j] = nsa[j] = nsb[j] = 0;
      if (active && g >= 0) {
        nx1[j] = base[g * gstride];
        nx2[j] = base[g * gstride + d.lanes];
        if (HAS_SRC) nsa[j] = load_src<real, st>(sa + (long long)g * d.lanes);
        if (HAS_SRC && TWO) nsb[j] = load_src<real, st>(sb + (long long)g * d.lanes);
      }
    }
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
      const int g = gb - j;
      if (g < 0) break;
      const GroupCoef<real> &k = tab[g];
      real x1, x2;
      const real y1 = A.template group<HAS_SRC>(k, cur1[j], cur2[j], csa[j], x1, x2);
      cnt += k.de * x1;
      if (HAS_R) {
        A.tsum = A.rho * k.q1 * y1 + k.decay * A.tsum;
        if (active) store_st<st, real>(ra + (long long)g * d.lanes, A.tsum * k.inv_de);
      }
      if (TWO) {
        real z1, z2;
        const real w1 = B.template group<HAS_SRC>(k, x1, x2, csb[j], z1, z2);
        if (HAS_R) {
          B.tsum = B.rho * k.q1 * w1 + k.decay * B.tsum;
          if (active) store_st<st, real>(rb + (long long)g * d.lanes, B.tsum * k.inv_de);
        }
        x1 = z1;
        x2 = z2;
      }
      if (active) {
        base[g * gstride] = x1;
        base[g * gstride + d.lanes] = x2;
      }
    }
#pragma unroll
    for (int j = 0; j < kUnroll; j++) {
      cur1[j] = nx1[j];
      cur2[j] = nx2[j];
      csa[j] = nsa[j];
      csb[j] = nsb[j];
    }
  }

  // reduce over the block's 8 angles and add to the voxel tallies
  red[0][threadIdx.y][threadIdx.x] = active ? (double)A.dep + (double)A.dep_c : 0.0;
  red[1][threadIdx.y][threadIdx.x] = active ? (double)cnt : 0.0;
  red[2][threadIdx.y][threadIdx.x] = (active && TWO) ? (double)B.dep + (double)B.dep_c : 0.0;
  __syncthreads();
  if (threadIdx.y == 0 && yz < d.nyz) {
    double sa_ = 0.0, sf = 0.0, sb_ = 0.0;
#pragma unroll
    for (int j = 0; j < kAnglesY; j++) {
      sa_ += red[0][j][threadIdx.x];
      sf += red[1][j][threadIdx.x];
      sb_ += red[2][j][threadIdx.x];
    }
    const double ra_ = (double)rho_a[yz];
    if (dose_a && ra_ > 0.0) atomicAdd(dose_a + yz, sa_ * dose_scale / ra_);
    if (flu) atomicAdd(flu + yz, sf * flu_scale);
    if (TWO) {
      const double rb_ = (double)rho_b[yz];
      if (dose_b && rb_ > 0.0) atomicAdd(dose_b + yz, sb_ * dose_scale / rb_);
    }
  }
}

}  // namespace

template <typename real, typename st>
cudaError_t launch_energy(const LaunchCtx &lc, const Dims &d, real *psi_k, const EnergyHalf<real, st> &ha,
                          const EnergyHalf<real, st> *hb, const GroupCoef<real> *coef, double *flu_yz,
                          double dose_scale, double flu_scale, const BeamStrides &bs, const StragCoef<real> *strag) {
  if constexpr (sizeof(real) == 4) {
    if (lc.energy_form == 1 && energy_f2_supported(d))
      return launch_energy_f2<st>(lc, d, psi_k, ha, hb, coef, flu_yz, dose_scale, flu_scale, bs, strag);
  }
  if (strag) return launch_energy_strag<real, st>(lc, d, psi_k, ha, hb, coef, strag, flu_yz, dose_scale, flu_scale, bs);
  const int ay = lc.energy_angles;
  dim3 block(kLanesX, ay);
  dim3 grid((d.nyz + kLanesX - 1) / kLanesX, (d.na + ay - 1) / ay, d.nbeam);
  const size_t smem = sizeof(GroupCoef<real>) * d.ng;
  const bool has_src = ha.src != nullptr, has_r = ha.r_out != nullptr;
  const EnergyHalf<real, st> &b = hb ? *hb : ha;
  auto go = [&](auto kern) -> cudaError_t {
    if (smem + sizeof(double) * 3 * 16 * kLanesX > 48 * 1024) {  // dynamic table + static reduction buffer
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, block, smem, lc.stream>>>(d, psi_k, ha.src, b.src, ha.r_out, b.r_out, ha.rho, b.rho, coef, ha.dose,
                                           b.dose, flu_yz, ha.c, b.c, dose_scale, flu_scale, bs);
    ++*lc.launches;
    return cudaGetLastError();
  };
  auto pick = [&](auto ay_tag) -> cudaError_t {
    constexpr int AY = decltype(ay_tag)::value;
#define PBS_E(S, R, T) \
  if (has_src == S && has_r == R && (hb != nullptr) == T) return go(k_energy<real, st, S, R, T, AY>);
    PBS_E(true, true, true) PBS_E(true, false, true) PBS_E(false, true, true) PBS_E(false, false, true)
    PBS_E(true, true, false) PBS_E(true, false, false) PBS_E(false, true, false) PBS_E(false, false, false)
#undef PBS_E
    return cudaErrorInvalidValue;
  };
  if (ay == 4) return pick(std::integral_constant<int, 4>{});
  if (ay == 8) return pick(std::integral_constant<int, 8>{});
  if (ay == 16) return pick(std::integral_constant<int, 16>{});
  return cudaErrorInvalidConfiguration;
}

template cudaError_t launch_energy<double, double>(const LaunchCtx &, const Dims &, double *,
                                                   const EnergyHalf<double, double> &,
                                                   const EnergyHalf<double, double> *, const GroupCoef<double> *,
                                                   double *, double, double, const BeamStrides &,
                                                   const StragCoef<double> *);
template cudaError_t launch_energy<float, float>(const LaunchCtx &, const Dims &, float *,
                                                 const EnergyHalf<float, float> &, const EnergyHalf<float, float> *,
                                                 const GroupCoef<float> *, double *, double, double, const BeamStrides &,
                                                 const StragCoef<float> *);
template cudaError_t launch_energy<float, __nv_bfloat16>(const LaunchCtx &, const Dims &, float *,
                                                         const EnergyHalf<float, __nv_bfloat16> &,
                                                         const EnergyHalf<float, __nv_bfloat16> *,
                                                         const GroupCoef<float> *, double *, double, double,
                                                         const BeamStrides &, const StragCoef<float> *);

}  // namespace pbs
