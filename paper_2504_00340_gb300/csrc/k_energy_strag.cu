// k_energy_strag.cu -- energy substep E(h) with energy straggling (Section
// 3.2, Eq. 0041-d with T != 0; Appendix A.2), one thread per lane
// (y, z, u, v), descending scan over the groups.
//
// The straggling term (rho/2) d^2(T psi)/dE^2 has two parts.  The drift
// (rho/2) d/dE(T' psi) is folded into the stopping power at the faces
// (S + T'/2) when the tables are built, so it runs through the same upwind
// blocks as S.  The interior-penalty part St (block tridiagonal: group g
// also sees psi_{g-1}) is taken explicitly inside the CN step, on the old
// state only:
//   (I - c A_S) x = (I + c A_S) psi + rho c St psi + c (src_old + src_new),
// so the system stays block upper-bidiagonal and one descending scan solves
// it; the only change to the scan is that group g reads psi_{g-1} one group
// ahead.  The deposited energy gains -rho c phi^T St psi.
//
// Two back-to-back substeps are fused as in k_energy.cu, but the second
// scan trails the first by one group: its explicit term at g needs the
// first scan's result at g - 1, which exists one iteration later.
#include "energy_scan.cuh"

#include <type_traits>

namespace pbs {

namespace {

using namespace escan;

constexpr int kLX = 32;  // lateral points per block (coalesced)
constexpr int kU = 4;    // groups per prefetch block

template <typename real>
struct Strag {
  real v[12];
  // 16-byte loads (the table is 256-byte aligned and 48 or 96 bytes a group);
  // every thread of a warp reads the same group: one broadcast per load
  __device__ __forceinline__ void load(const StragCoef<real> *p) {
    if constexpr (sizeof(real) == 4) {
      const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
      for (int i = 0; i < 3; i++) {
        const float4 t = __ldg(q + i);
        v[4 * i] = t.x;
        v[4 * i + 1] = t.y;
        v[4 * i + 2] = t.z;
        v[4 * i + 3] = t.w;
      }
    } else {
      const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
      for (int i = 0; i < 6; i++) {
        const double2 t = __ldg(q + i);
        v[2 * i] = t.x;
        v[2 * i + 1] = t.y;
      }
    }
  }
  // (e0, e1) = lo l + d o + up u
  __device__ __forceinline__ void apply(real l1, real l2, real o1, real o2, real u1, real u2, real &e0,
                                        real &e1) const {
    e0 = v[0] * l1 + v[1] * l2 + v[4] * o1 + v[5] * o2 + v[8] * u1 + v[9] * u2;
    e1 = v[2] * l1 + v[3] * l2 + v[6] * o1 + v[7] * o2 + v[10] * u1 + v[11] * u2;
  }
};

template <typename real, typename st, bool HAS_SRC, bool HAS_R, bool TWO, int kAY>
__global__ void __launch_bounds__(kLX *kAY)
    k_energy_strag(Dims d, real *__restrict__ psi, const st *__restrict__ src_a, const st *__restrict__ src_b,
                   st *__restrict__ r_a, st *__restrict__ r_b, const real *__restrict__ rho_a,
                   const real *__restrict__ rho_b, const GroupCoef<real> *__restrict__ coef,
                   const StragCoef<real> *__restrict__ strag, double *__restrict__ dose_a,
                   double *__restrict__ dose_b, double *__restrict__ flu, real c_a, real c_b, double dose_scale,
                   double flu_scale, BeamStrides bs) {
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
  const int tid = threadIdx.y * kLX + threadIdx.x;
  for (int g = tid; g < d.ng; g += kLX * kAY) tab[g] = coef[g];
  __shared__ double red[3][kAY][kLX];
  __syncthreads();

  const int yz = blockIdx.x * kLX + threadIdx.x;
  const int a = blockIdx.y * kAY + threadIdx.y;
  const bool active = (yz < d.nyz) && (a < d.na);
  const long long lane = (long long)a * d.nyz + yz;
  const long long gstride = 2 * d.lanes;

  Scan<real> A, B;
  A.init(active ? rho_a[yz] : real(0), c_a);
  if (TWO) B.init(active ? rho_b[yz] : real(0), c_b);
  real cnt = 0;

  real *base = psi + lane;
  const st *sa = HAS_SRC ? src_a + lane : nullptr;
  const st *sb = (HAS_SRC && TWO) ? src_b + lane : nullptr;
  st *ra = HAS_R ? r_a + lane : nullptr;
  st *rb = (HAS_R && TWO) ? r_b + lane : nullptr;

  real cur1[kU], cur2[kU], csa[kU], csb[kU];
  real nx1[kU], nx2[kU], nsa[kU], nsb[kU];
  const int G = d.ng;
#pragma unroll
  for (int j = 0; j < kU; j++) {
    const int g = G - 1 - j;
    cur1[j] = cur2[j] = csa[j] = csb[j] = 0;
    if (active && g >= 0) {
      cur1[j] = base[g * gstride];
      cur2[j] = base[g * gstride + d.lanes];
      if (HAS_SRC) csa[j] = load_src<real, st>(sa + (long long)g * d.lanes);
      if (HAS_SRC && TWO) csb[j] = load_src<real, st>(sb + (long long)g * d.lanes);
    }
  }
  real op1 = 0, op2 = 0;  // old psi at g + 1 (first scan)
  // second scan, one group behind: the first scan's results at g + 1 and
  // g + 2, and the second substep's source at g + 1
  real mc1 = 0, mc2 = 0, mu1 = 0, mu2 = 0, sbc = 0;

  // second scan at group gq, lower neighbour (l1, l2) of the first scan's result
  auto second = [&](int gq, real l1, real l2) {
    const GroupCoef<real> &k = tab[gq];
    Strag<real> sc;
    sc.load(strag + gq);
    real e0, e1, z1, z2;
    sc.apply(l1, l2, mc1, mc2, mu1, mu2, e0, e1);
    const real w1 = B.template group_x<HAS_SRC>(k, mc1, mc2, sbc, e0, e1, z1, z2);
    if (HAS_R) {
      B.tsum = B.rho * k.q1 * w1 + k.decay * B.tsum;
      if (active) store_st<st, real>(rb + (long long)gq * d.lanes, B.tsum * k.inv_de);
    }
    if (active) {
      base[gq * gstride] = z1;
      base[gq * gstride + d.lanes] = z2;
    }
  };

  for (int gb = G - 1; gb >= 0; gb -= kU) {
#pragma unroll
    for (int j = 0; j < kU; j++) {
      const int g = gb - kU - j;
      nx1[j] = nx2[j] = nsa[j] = nsb[j] = 0;
      if (active && g >= 0) {
        nx1[j] = base[g * gstride];
        nx2[j] = base[g * gstride + d.lanes];
        if (HAS_SRC) nsa[j] = load_src<real, st>(sa + (long long)g * d.lanes);
        if (HAS_SRC && TWO) nsb[j] = load_src<real, st>(sb + (long long)g * d.lanes);
      }
    }
#pragma unroll
    for (int j = 0; j < kU; j++) {
      const int g = gb - j;
      if (g < 0) break;
      const GroupCoef<real> &k = tab[g];
      Strag<real> sc;
      sc.load(strag + g);
      // old psi at g - 1: the next register of this block, or the first of the next block (0 below g = 0)
      const real l1 = (j + 1 < kU) ? cur1[j + 1] : nx1[0];
      const real l2 = (j + 1 < kU) ? cur2[j + 1] : nx2[0];
      real e0, e1, x1, x2;
      sc.apply(l1, l2, cur1[j], cur2[j], op1, op2, e0, e1);
      const real y1 = A.template group_x<HAS_SRC>(k, cur1[j], cur2[j], csa[j], e0, e1, x1, x2);
      cnt += k.de * x1;
      if (HAS_R) {
        A.tsum = A.rho * k.q1 * y1 + k.decay * A.tsum;
        if (active) store_st<st, real>(ra + (long long)g * d.lanes, A.tsum * k.inv_de);
      }
      op1 = cur1[j];
      op2 = cur2[j];
      if (TWO) {
        if (g + 1 < G) second(g + 1, x1, x2);
        mu1 = mc1;
        mu2 = mc2;
        mc1 = x1;
        mc2 = x2;
        sbc = csb[j];
      } else if (active) {
        base[g * gstride] = x1;
        base[g * gstride + d.lanes] = x2;
      }
    }
#pragma unroll
    for (int j = 0; j < kU; j++) {
      cur1[j] = nx1[j];
      cur2[j] = nx2[j];
      csa[j] = nsa[j];
      csb[j] = nsb[j];
    }
  }
  if (TWO && G > 0) second(0, real(0), real(0));

  red[0][threadIdx.y][threadIdx.x] = active ? (double)A.dep + (double)A.dep_c : 0.0;
  red[1][threadIdx.y][threadIdx.x] = active ? (double)cnt : 0.0;
  red[2][threadIdx.y][threadIdx.x] = (active && TWO) ? (double)B.dep + (double)B.dep_c : 0.0;
  __syncthreads();
  if (threadIdx.y == 0 && yz < d.nyz) {
    double sa_ = 0.0, sf = 0.0, sb_ = 0.0;
#pragma unroll
    for (int j = 0; j < kAY; j++) {
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
cudaError_t launch_energy_strag(const LaunchCtx &lc, const Dims &d, real *psi_k, const EnergyHalf<real, st> &ha,
                                const EnergyHalf<real, st> *hb, const GroupCoef<real> *coef,
                                const StragCoef<real> *strag, double *flu_yz, double dose_scale, double flu_scale,
                                const BeamStrides &bs) {
  const int ay = lc.energy_angles;
  dim3 block(kLX, ay);
  dim3 grid((d.nyz + kLX - 1) / kLX, (d.na + ay - 1) / ay, d.nbeam);
  const size_t smem = sizeof(GroupCoef<real>) * d.ng;
  const bool has_src = ha.src != nullptr, has_r = ha.r_out != nullptr;
  const EnergyHalf<real, st> &b = hb ? *hb : ha;
  auto go = [&](auto kern) -> cudaError_t {
    if (smem + sizeof(double) * 3 * 16 * kLX > 48 * 1024) {  // dynamic table + static reduction buffer
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    kern<<<grid, block, smem, lc.stream>>>(d, psi_k, ha.src, b.src, ha.r_out, b.r_out, ha.rho, b.rho, coef, strag,
                                           ha.dose, b.dose, flu_yz, ha.c, b.c, dose_scale, flu_scale, bs);
    ++*lc.launches;
    return cudaGetLastError();
  };
  auto pick = [&](auto ay_tag) -> cudaError_t {
    constexpr int AY = decltype(ay_tag)::value;
#define PBS_E(S, R, T) \
  if (has_src == S && has_r == R && (hb != nullptr) == T) return go(k_energy_strag<real, st, S, R, T, AY>);
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

template cudaError_t launch_energy_strag<double, double>(const LaunchCtx &, const Dims &, double *,
                                                         const EnergyHalf<double, double> &,
                                                         const EnergyHalf<double, double> *, const GroupCoef<double> *,
                                                         const StragCoef<double> *, double *, double, double,
                                                         const BeamStrides &);
template cudaError_t launch_energy_strag<float, float>(const LaunchCtx &, const Dims &, float *,
                                                       const EnergyHalf<float, float> &,
                                                       const EnergyHalf<float, float> *, const GroupCoef<float> *,
                                                       const StragCoef<float> *, double *, double, double,
                                                       const BeamStrides &);
template cudaError_t launch_energy_strag<float, __nv_bfloat16>(const LaunchCtx &, const Dims &, float *,
                                                               const EnergyHalf<float, __nv_bfloat16> &,
                                                               const EnergyHalf<float, __nv_bfloat16> *,
                                                               const GroupCoef<float> *, const StragCoef<float> *,
                                                               double *, double, double, const BeamStrides &);

}  // namespace pbs
