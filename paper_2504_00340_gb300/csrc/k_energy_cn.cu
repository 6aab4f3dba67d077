// k_energy_cn.cu -- energy substep E(h) with energy straggling taken fully
// into the Crank-Nicolson step (Section 3.3 applied to the whole L3/L4 of
// Eq. 0041-do, straggling included; pbs_options.straggling_integrator = 1).
//
// With the interior-penalty straggling blocks the per-lane system
//   (I - c A) x = (I + c A) psi + c (src_old + src_new),   A = A_S + A_T,
// is block tridiagonal:  L_g x_{g-1} + D_g x_g + U_g x_{g+1} = rhs_g  with
//   L_g = -c A_T,lo(g),  D_g = I - c (A_S,gg + A_T,gg),  U_g = -c (A_S,up + A_T,up).
// Block elimination from the top group down and substitution upward:
//   D'_{G-1} = D_{G-1},  D'_g = D_g - U_g D'^{-1}_{g+1} L_{g+1},
//   b'_{G-1} = rhs_{G-1}, b'_g = rhs_g - U_g D'^{-1}_{g+1} b'_{g+1},
//   x_0 = D'^{-1}_0 b'_0,  x_g = D'^{-1}_g (b'_g - L_g x_{g-1}).
// Every block is rho c times a per-unit-density table, so D'^{-1} depends on
// the lateral point only (not on the angle): k_cn_factor computes it once
// per substep and lateral point into a [g][4][yz] scratch region; the angle
// lanes then run two streaming passes over psi:
//   pass A (descending): right-hand side (psi_{g-1} read one group ahead),
//     elimination, b' stored in place of psi;
//   pass B (ascending): substitution, x stored in place of b'.
// The deposited energy is the operator form -phi^T c A (psi + x) - c phi^T src,
// accumulated as columns: -rho c sum_g Om_g . (psi_g + x_g) with the column
// weights Om = (A / (rho c))^T phi tabulated per group (pass A adds the psi
// half, pass B the x half).  The energy-summed source input of the next
// component, R_g = T_g / dE_g with T_g = w_g + decay_g T_{g+1} and
// w_g = rho q1_g (psi^1 + x^1)_g, needs the descending order: pass A stores
// rho q1 psi^1, pass B adds rho q1 x^1, and k_cn_r runs the recursion.
#include "energy_scan.cuh"

namespace pbs {

namespace {

using namespace escan;

constexpr int kLX = 32;  // lateral points per block (coalesced)

template <typename real>
__device__ __forceinline__ void load12(const StragCoef<real> *p, real (&v)[12]) {
  const real *q = reinterpret_cast<const real *>(p);
#pragma unroll
  for (int i = 0; i < 12; i++) v[i] = __ldg(q + i);
}

// 2x2 helpers, row-major [r][q] -> m[2 r + q]
template <typename real>
__device__ __forceinline__ void mv2(const real (&m)[4], real x0, real x1, real &y0, real &y1) {
  y0 = m[0] * x0 + m[1] * x1;
  y1 = m[2] * x0 + m[3] * x1;
}

// Blocks of row g for density rho and CN factor c (rc = rho c, ht = rc / 2):
// c A_S,gg, c A_S,up (from the stopping-power table) and the straggling ones.
template <typename real>
struct RowBlocks {
  real sgg[4], sup[4], tlo[4], tgg[4], tup[4];
  __device__ __forceinline__ void make(const GroupCoef<real> &k, const real (&st)[12], real rc, bool has_up) {
    const real am = rc * k.sm, ap = rc * k.sp, sg = rc * k.sig, ht = real(0.5) * rc;
    sgg[0] = -am - sg;
    sgg[1] = am;
    sgg[2] = real(-3) * ap;
    sgg[3] = -ap - real(2) * am - sg;
    const real a = has_up ? ap : real(0);
    sup[0] = a;
    sup[1] = -a;
    sup[2] = real(3) * a;
    sup[3] = real(-3) * a;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      tlo[i] = ht * st[i];
      tgg[i] = ht * st[4 + i];
      tup[i] = ht * st[8 + i];
    }
  }
};

// D'^{-1} per (g, lateral point): one thread per lateral point, groups from the top.
template <typename real>
__global__ void __launch_bounds__(256) k_cn_factor(Dims d, const real *__restrict__ rho,
                                                   const GroupCoef<real> *__restrict__ coef,
                                                   const StragCoef<real> *__restrict__ strag, real c,
                                                   real *__restrict__ dinv) {
  const int yz = blockIdx.x * blockDim.x + threadIdx.x;
  if (yz >= d.nyz) return;
  const real rc = rho[yz] * c;
  const long long gs = 4LL * d.nyz;
  real ln[4] = {0, 0, 0, 0};      // L_{g+1}
  real di[4] = {0, 0, 0, 0};      // D'^{-1}_{g+1}
  for (int g = d.ng - 1; g >= 0; g--) {
    real st[12];
    load12(strag + g, st);
    RowBlocks<real> b;
    b.make(coef[g], st, rc, g + 1 < d.ng);
    real D[4], U[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
      D[i] = ((i == 0 || i == 3) ? real(1) : real(0)) - b.sgg[i] - b.tgg[i];
      U[i] = -b.sup[i] - b.tup[i];
    }
    if (g + 1 < d.ng) {
      // W = U D'^{-1}_{g+1};  D -= W L_{g+1}
      real W[4];
      W[0] = U[0] * di[0] + U[1] * di[2];
      W[1] = U[0] * di[1] + U[1] * di[3];
      W[2] = U[2] * di[0] + U[3] * di[2];
      W[3] = U[2] * di[1] + U[3] * di[3];
      D[0] -= W[0] * ln[0] + W[1] * ln[2];
      D[1] -= W[0] * ln[1] + W[1] * ln[3];
      D[2] -= W[2] * ln[0] + W[3] * ln[2];
      D[3] -= W[2] * ln[1] + W[3] * ln[3];
    }
    const real inv = real(1) / (D[0] * D[3] - D[1] * D[2]);
    di[0] = D[3] * inv;
    di[1] = -D[1] * inv;
    di[2] = -D[2] * inv;
    di[3] = D[0] * inv;
    real *o = dinv + g * gs + yz;
#pragma unroll
    for (int i = 0; i < 4; i++) o[(long long)i * d.nyz] = di[i];
#pragma unroll
    for (int i = 0; i < 4; i++) ln[i] = -b.tlo[i];
  }
}

template <typename real>
__device__ __forceinline__ void load_dinv(const real *dinv, int g, int yz, long long nyz, real (&m)[4]) {
  const real *p = dinv + (long long)g * 4 * nyz + yz;
#pragma unroll
  for (int i = 0; i < 4; i++) m[i] = p[(long long)i * nyz];
}

// Pass A: right-hand side and elimination, descending.
template <typename real, typename st, bool HAS_SRC, bool HAS_R, int kAY>
__global__ void __launch_bounds__(kLX *kAY)
    k_cn_a(Dims d, real *__restrict__ psi, const st *__restrict__ src, st *__restrict__ r_out,
           const real *__restrict__ rho, const GroupCoef<real> *__restrict__ coef,
           const StragCoef<real> *__restrict__ strag, const real *__restrict__ omega, const real *__restrict__ dinv,
           double *__restrict__ dose, real c, double dose_scale, BeamStrides bs) {
  {
    const long long b = blockIdx.z;
    psi += b * bs.psi;
    if (HAS_SRC) src += b * bs.src;
    if (HAS_R) r_out += b * bs.src;
    if (dose) dose += b * bs.dose;
  }
  __shared__ double red[kAY][kLX];
  const int yz = blockIdx.x * kLX + threadIdx.x;
  const int a = blockIdx.y * kAY + threadIdx.y;
  const bool active = (yz < d.nyz) && (a < d.na);
  const long long lane = (long long)a * d.nyz + yz;
  const long long gstride = 2 * d.lanes;
  const int G = d.ng;
  const real rc = active ? rho[yz] * c : real(0);
  real *base = psi + lane;
  real dep = 0, dep_c = 0;
  real o1 = 0, o2 = 0, l1 = 0, l2 = 0;  // psi_g and psi_{g-1}
  real u1 = 0, u2 = 0;                  // psi_{g+1}
  real bp1 = 0, bp2 = 0;                // b'_{g+1}
  if (active) {
    o1 = base[(G - 1) * gstride];
    o2 = base[(G - 1) * gstride + d.lanes];
  }
  for (int g = G - 1; g >= 0; g--) {
    l1 = l2 = 0;
    if (active && g > 0) {
      l1 = base[(g - 1) * gstride];
      l2 = base[(g - 1) * gstride + d.lanes];
    }
    const GroupCoef<real> k = coef[g];
    real stc[12];
    load12(strag + g, stc);
    RowBlocks<real> b;
    b.make(k, stc, rc, g + 1 < G);
    // rhs = psi + c A psi + c src
    real r0 = o1 + b.sgg[0] * o1 + b.sgg[1] * o2 + b.sup[0] * u1 + b.sup[1] * u2 + b.tlo[0] * l1 + b.tlo[1] * l2 +
              b.tgg[0] * o1 + b.tgg[1] * o2 + b.tup[0] * u1 + b.tup[1] * u2;
    real r1 = o2 + b.sgg[2] * o1 + b.sgg[3] * o2 + b.sup[2] * u1 + b.sup[3] * u2 + b.tlo[2] * l1 + b.tlo[3] * l2 +
              b.tgg[2] * o1 + b.tgg[3] * o2 + b.tup[2] * u1 + b.tup[3] * u2;
    real s = 0;
    if (HAS_SRC) {
      s = active ? load_src<real, st>(src + (long long)g * d.lanes + lane) : real(0);
      r0 += c * s;
    }
    if (g + 1 < G) {  // b' = rhs - U D'^{-1}_{g+1} b'_{g+1}
      real di[4], z0, z1;
      load_dinv(dinv, g + 1, active ? yz : 0, d.nyz, di);
      mv2(di, bp1, bp2, z0, z1);
      r0 += (b.sup[0] + b.tup[0]) * z0 + (b.sup[1] + b.tup[1]) * z1;
      r1 += (b.sup[2] + b.tup[2]) * z0 + (b.sup[3] + b.tup[3]) * z1;
    }
    // deposited energy: the psi half of the column form, and the source term
    const real om0 = omega[2 * g], om1 = omega[2 * g + 1];
    real t = rc * (om0 * o1 + om1 * o2);
    if (HAS_SRC) t += c * k.ehat * s;
    comp_add(dep, dep_c, -t);
    if (active) {
      base[g * gstride] = r0;
      base[g * gstride + d.lanes] = r1;
      if (HAS_R) store_st<st, real>(r_out + (long long)g * d.lanes + lane, rho[yz] * k.q1 * o1);
    }
    bp1 = r0;
    bp2 = r1;
    u1 = o1;
    u2 = o2;
    o1 = l1;
    o2 = l2;
  }
  red[threadIdx.y][threadIdx.x] = active ? (double)dep + (double)dep_c : 0.0;
  __syncthreads();
  if (threadIdx.y == 0 && yz < d.nyz) {
    double sa = 0.0;
#pragma unroll
    for (int j = 0; j < kAY; j++) sa += red[j][threadIdx.x];
    const double r_ = (double)rho[yz];
    if (dose && r_ > 0.0) atomicAdd(dose + yz, sa * dose_scale / r_);
  }
}

// Pass B: substitution, ascending; the x half of the dose, fluence, R input.
template <typename real, typename st, bool HAS_R, int kAY>
__global__ void __launch_bounds__(kLX *kAY)
    k_cn_b(Dims d, real *__restrict__ psi, st *__restrict__ r_out, const real *__restrict__ rho,
           const GroupCoef<real> *__restrict__ coef, const StragCoef<real> *__restrict__ strag,
           const real *__restrict__ omega, const real *__restrict__ dinv, double *__restrict__ dose,
           double *__restrict__ flu, real c, double dose_scale, double flu_scale, BeamStrides bs) {
  {
    const long long b = blockIdx.z;
    psi += b * bs.psi;
    if (HAS_R) r_out += b * bs.src;
    if (dose) dose += b * bs.dose;
    if (flu) flu += b * bs.flu;
  }
  __shared__ double red[2][kAY][kLX];
  const int yz = blockIdx.x * kLX + threadIdx.x;
  const int a = blockIdx.y * kAY + threadIdx.y;
  const bool active = (yz < d.nyz) && (a < d.na);
  const long long lane = (long long)a * d.nyz + yz;
  const long long gstride = 2 * d.lanes;
  const int G = d.ng;
  const real rc = active ? rho[yz] * c : real(0);
  const real ht = real(0.5) * rc;
  real *base = psi + lane;
  real dep = 0, dep_c = 0, cnt = 0;
  real xp1 = 0, xp2 = 0;  // x_{g-1}
  for (int g = 0; g < G; g++) {
    real b1 = 0, b2 = 0;
    if (active) {
      b1 = base[g * gstride];
      b2 = base[g * gstride + d.lanes];
    }
    if (g > 0) {  // b' - L_g x_{g-1},  L_g = -ht lo_g
      real stc[12];
      load12(strag + g, stc);
      b1 += ht * (stc[0] * xp1 + stc[1] * xp2);
      b2 += ht * (stc[2] * xp1 + stc[3] * xp2);
    }
    real di[4], x1, x2;
    load_dinv(dinv, g, active ? yz : 0, d.nyz, di);
    mv2(di, b1, b2, x1, x2);
    const GroupCoef<real> k = coef[g];
    comp_add(dep, dep_c, -rc * (omega[2 * g] * x1 + omega[2 * g + 1] * x2));
    cnt += k.de * x1;
    if (active) {
      base[g * gstride] = x1;
      base[g * gstride + d.lanes] = x2;
      if (HAS_R) {
        st *rp = r_out + (long long)g * d.lanes + lane;
        store_st<st, real>(rp, load_src<real, st>(rp) + rho[yz] * k.q1 * x1);
      }
    }
    xp1 = x1;
    xp2 = x2;
  }
  red[0][threadIdx.y][threadIdx.x] = active ? (double)dep + (double)dep_c : 0.0;
  red[1][threadIdx.y][threadIdx.x] = active ? (double)cnt : 0.0;
  __syncthreads();
  if (threadIdx.y == 0 && yz < d.nyz) {
    double sa = 0.0, sf = 0.0;
#pragma unroll
    for (int j = 0; j < kAY; j++) {
      sa += red[0][j][threadIdx.x];
      sf += red[1][j][threadIdx.x];
    }
    const double r_ = (double)rho[yz];
    if (dose && r_ > 0.0) atomicAdd(dose + yz, sa * dose_scale / r_);
    if (flu) atomicAdd(flu + yz, sf * flu_scale);
  }
}

// R recursion in place, descending: T_g = w_g + decay_g T_{g+1}, R_g = T_g / dE_g.
template <typename real, typename st>
__global__ void __launch_bounds__(256) k_cn_r(Dims d, st *__restrict__ r, const GroupCoef<real> *__restrict__ coef,
                                              BeamStrides bs) {
  const long long lane = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (lane >= d.lanes) return;
  st *p = r + blockIdx.y * bs.src + lane;
  real t = 0;
  for (int g = d.ng - 1; g >= 0; g--) {
    const GroupCoef<real> k = coef[g];
    t = load_src<real, st>(p + (long long)g * d.lanes) + k.decay * t;
    store_st<st, real>(p + (long long)g * d.lanes, t * k.inv_de);
  }
}

}  // namespace

template <typename real>
cudaError_t launch_cn_factor(const LaunchCtx &lc, const Dims &d, const real *rho, const GroupCoef<real> *coef,
                             const StragCoef<real> *strag, real c, real *dinv) {
  k_cn_factor<real><<<(d.nyz + 255) / 256, 256, 0, lc.stream>>>(d, rho, coef, strag, c, dinv);
  ++*lc.launches;
  return cudaGetLastError();
}

template <typename real, typename st>
cudaError_t launch_energy_cn(const LaunchCtx &lc, const Dims &d, real *psi_k, const EnergyHalf<real, st> &h,
                             const GroupCoef<real> *coef, const StragCoef<real> *strag, const real *omega,
                             const real *dinv, double *flu_yz, double dose_scale, double flu_scale,
                             const BeamStrides &bs) {
  constexpr int AY = 8;
  dim3 block(kLX, AY);
  dim3 grid((d.nyz + kLX - 1) / kLX, (d.na + AY - 1) / AY, d.nbeam);
  const bool has_src = h.src != nullptr, has_r = h.r_out != nullptr;
  if (has_src && has_r)
    k_cn_a<real, st, true, true, AY><<<grid, block, 0, lc.stream>>>(d, psi_k, h.src, h.r_out, h.rho, coef, strag,
                                                                     omega, dinv, h.dose, h.c, dose_scale, bs);
  else if (has_src)
    k_cn_a<real, st, true, false, AY><<<grid, block, 0, lc.stream>>>(d, psi_k, h.src, h.r_out, h.rho, coef, strag,
                                                                      omega, dinv, h.dose, h.c, dose_scale, bs);
  else if (has_r)
    k_cn_a<real, st, false, true, AY><<<grid, block, 0, lc.stream>>>(d, psi_k, h.src, h.r_out, h.rho, coef, strag,
                                                                      omega, dinv, h.dose, h.c, dose_scale, bs);
  else
    k_cn_a<real, st, false, false, AY><<<grid, block, 0, lc.stream>>>(d, psi_k, h.src, h.r_out, h.rho, coef, strag,
                                                                       omega, dinv, h.dose, h.c, dose_scale, bs);
  ++*lc.launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (has_r)
    k_cn_b<real, st, true, AY><<<grid, block, 0, lc.stream>>>(d, psi_k, h.r_out, h.rho, coef, strag, omega, dinv,
                                                               h.dose, flu_yz, h.c, dose_scale, flu_scale, bs);
  else
    k_cn_b<real, st, false, AY><<<grid, block, 0, lc.stream>>>(d, psi_k, h.r_out, h.rho, coef, strag, omega, dinv,
                                                                h.dose, flu_yz, h.c, dose_scale, flu_scale, bs);
  ++*lc.launches;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (has_r) {
    dim3 rg((unsigned)((d.lanes + 255) / 256), (unsigned)d.nbeam);
    k_cn_r<real, st><<<rg, 256, 0, lc.stream>>>(d, h.r_out, coef, bs);
    ++*lc.launches;
    e = cudaGetLastError();
  }
  return e;
}

template cudaError_t launch_cn_factor<double>(const LaunchCtx &, const Dims &, const double *,
                                              const GroupCoef<double> *, const StragCoef<double> *, double, double *);
template cudaError_t launch_cn_factor<float>(const LaunchCtx &, const Dims &, const float *, const GroupCoef<float> *,
                                             const StragCoef<float> *, float, float *);
template cudaError_t launch_energy_cn<double, double>(const LaunchCtx &, const Dims &, double *,
                                                      const EnergyHalf<double, double> &, const GroupCoef<double> *,
                                                      const StragCoef<double> *, const double *, const double *,
                                                      double *, double, double, const BeamStrides &);
template cudaError_t launch_energy_cn<float, float>(const LaunchCtx &, const Dims &, float *,
                                                    const EnergyHalf<float, float> &, const GroupCoef<float> *,
                                                    const StragCoef<float> *, const float *, const float *, double *,
                                                    double, double, const BeamStrides &);
template cudaError_t launch_energy_cn<float, __nv_bfloat16>(const LaunchCtx &, const Dims &, float *,
                                                            const EnergyHalf<float, __nv_bfloat16> &,
                                                            const GroupCoef<float> *, const StragCoef<float> *,
                                                            const float *, const float *, double *, double, double,
                                                            const BeamStrides &);

}  // namespace pbs
