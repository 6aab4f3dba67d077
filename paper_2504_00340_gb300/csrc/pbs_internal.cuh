// pbs_internal.cuh -- device-side definitions shared by the library's kernels.
//
// Layout of the device workspace (one context):
//   psi   [k][g][c][a][p][q]      (K+1) components, real = double or float
//   rbuf  2 x [g][a][p][q]        energy-summed catastrophic source input R (K>0),
//                                 one per E substep of a fused pair
//   sbuf  2 x [g][a][p][q]        catastrophic source src = du dv P2_g R  (K>0)
//   rho   [s][p][q]               density per depth slab, real
//   dose  [s][p][q]               FP64 dose tally
//   flu   [s][p][q]               FP64 planar fluence at depth s*dx
//   coef  [g]                     GroupCoef<real>
//   ts    [g]                     group-averaged scattering power, real
//   p2    [g][a][a']              P^2 densities (source storage type)
//   err   int[4]                  device status word (timeouts)
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace pbs {

constexpr int kMaxAngle = 16;  // nu, nv <= 16 on the device path

// Per-group energy coefficients, per unit density (multiply by rho).
template <typename real>
struct GroupCoef {
  real sm;      // S_{g-1/2} / dE_g
  real sp;      // S_{g+1/2} / dE_g
  real sig;     // sigma_ct (mass)
  real ehat;    // E_g dE_g        (energy-content weight of psi^1)
  real dq;      // dE_g^2 / 6      (energy-content weight of psi^2)
  real de;      // dE_g            (particle-count weight of psi^1)
  real inv_de;  // 1 / dE_g
  real q1;      // lambda sigma_g dE_g / Z_g   (source weight of group g as emitter)
  real decay;   // exp(-lambda (E_{g+1} - E_g)), 0 for the top group
  real pad;
};

// Energy straggling (interior-penalty DG, Section 3.2): the 2x2 blocks of
// group g on psi_{g-1}, psi_g, psi_{g+1}, per unit density and times 2, so
// that rho c (lo psi_{g-1} + d psi_g + up psi_{g+1}) is the explicit
// straggling contribution of a substep with CN factor c = h/2.  Row-major
// [r][q]: entry [2 r + q] couples DG coefficient q to row r.
template <typename real>
struct StragCoef {
  real lo[4], d[4], up[4];
};

struct Dims {
  int ny, nz, ng, nu, nv, na, nyz, ncomp;  // ncomp = n_beams * (K + 1): all components
  int nbeam;                                // independent beams
  long long lanes;                          // na * nyz
  long long comp_elems;                     // ng * 2 * lanes
};

// Device status word: slot 0 counts timeouts, slot 1 records where.
enum : int { kErrTimeoutSourceMma = 2, kErrTimeoutAngular = 3, kErrTimeoutBatch = 4 };

// ----------------------------------------------------------------------------
// PTX helpers: shared-memory addresses, mbarriers, 1-D bulk (TMA) copies.
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of an mbarrier to complete, giving up after about
// `max_cycles` SM clocks.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long max_cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > max_cycles) return false;
  }
  return true;
}

// Bulk copy global -> shared (async proxy), completion signalled on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ----------------------------------------------------------------------------
// Superbee-limited slope and upwind face flux (Section 3.4, Eq. distansport).
// slope(a, b) equals b * eta(a / b) with eta(t) = max[0, min(2t,1), min(t,2)]
// wherever a / b is defined; written without the division:
//   opposite signs or a zero  ->  0,   otherwise  sign(b) * min(max|.|, 2 min|.|).
// ----------------------------------------------------------------------------
// Sign agreement from the sign bits: a product a*b can underflow to zero in
// FP32 for tiny (but still representable) differences.
__device__ __forceinline__ bool same_sign(float a, float b) {
  return ((__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u) == 0u;
}
__device__ __forceinline__ bool same_sign(double a, double b) {
  return ((__double_as_longlong(a) ^ __double_as_longlong(b)) & (long long)0x8000000000000000ULL) == 0;
}

template <typename real>
__device__ __forceinline__ real superbee_slope(real a, real b) {
  real aa = fabs(a), ab = fabs(b);
  real m = fmin(fmax(aa, ab), real(2) * fmin(aa, ab));  // zero if a or b is zero
  return same_sign(a, b) ? copysign(m, b) : real(0);
}

// Flux through the face between cells p0 (left) and p1 (right) for speed s:
//   s > 0:  s (p0 + slope(p0 - pm1, p1 - p0) / 2)
//   s < 0:  s (p1 - slope(p2 - p1, p1 - p0) / 2)
template <typename real>
__device__ __forceinline__ real face_flux(bool pos, real s, real pm1, real p0, real p1, real p2) {
  real b = p1 - p0;
  return pos ? s * (p0 + real(0.5) * superbee_slope(p0 - pm1, b))
             : s * (p1 - real(0.5) * superbee_slope(p2 - p1, b));
}

// ----------------------------------------------------------------------------
// Kernel launchers (defined in the k_*.cu files).
// ----------------------------------------------------------------------------
struct LaunchCtx {
  cudaStream_t stream;
  int num_sms;
  long long *launches;  // host counter
  int *err = nullptr;   // device status word (bounded waits record timeouts here)
  // launch shapes chosen by the autotuner (pbs_autotune)
  int energy_angles = 8;   // energy: angles per block (4, 8 or 16) x 32 lateral points
  int transport_ctas = 0;  // streaming transport: resident CTAs per SM (0 = as many as fit)
  int transport_cols = 0;  // streaming transport: columns per lane, 4 or 6 (0 = by row width)
  int angular_form = 5;    // angular substep: 0 direct, 1 TMA-staged persistent, 2-7 packed FP32x2
                           // (2 as compiled, 3 at 64 registers, 4 two stacks per CTA; where the grid allows, else 0)
  int energy_form = 1;     // FP32 energy substep: 0 one lane per thread, 1 packed FP32x2
                           // (form 1 where the grid allows, else 0)
  int source_form = 1;     // BF16 source contraction: 0 tile by tile, 1 TMA/MMA/epilogue pipeline
  int angular_exact = 0;   // angular time integrator: 0 Crank-Nicolson, 1 exact exponential per mode
  int transport_cn = 0;    // transport time integrator: 0 explicit trapezoid, 1 CN with lagged slope
};

// One E substep's per-lane inputs and outputs: density of its slab, c = h/2,
// source of this component (sum of the trapezoid ends, or NULL), energy-summed
// source input R for the next component (or NULL), dose slab.
template <typename real, typename st>
struct EnergyHalf {
  const real *rho;
  real c;
  const st *src;
  st *r_out;
  double *dose;
};

// Per-beam strides of the pointers an energy launch receives (blockIdx.z =
// beam): psi of the same component of the next beam, its source/R buffers,
// its dose slab array and its fluence plane array.
struct BeamStrides {
  long long psi, src, dose, flu;
};

bool energy_f2_supported(const Dims &d);
template <typename st>
cudaError_t launch_energy_f2(const LaunchCtx &lc, const Dims &d, float *psi_k, const EnergyHalf<float, st> &ha,
                             const EnergyHalf<float, st> *hb, const GroupCoef<float> *coef, double *flu_yz,
                             double dose_scale, double flu_scale, const BeamStrides &bs,
                             const StragCoef<float> *strag = nullptr);

// E substep on one component of every beam; with hb != NULL, two consecutive
// E substeps (ha then hb) fused in one pass.  flu_yz receives the fluence
// after ha.
template <typename real, typename st>
cudaError_t launch_energy(const LaunchCtx &lc, const Dims &d, real *psi_k, const EnergyHalf<real, st> &ha,
                          const EnergyHalf<real, st> *hb, const GroupCoef<real> *coef, double *flu_yz,
                          double dose_scale, double flu_scale, const BeamStrides &bs,
                          const StragCoef<real> *strag = nullptr);

// E substep with straggling inside the CN step (k_energy_cn.cu): the
// eliminated diagonal blocks D'^{-1} of a slab ([g][4][yz]), then the two
// passes over one component (and the R recursion when h.r_out is set).
template <typename real>
cudaError_t launch_cn_factor(const LaunchCtx &lc, const Dims &d, const real *rho, const GroupCoef<real> *coef,
                             const StragCoef<real> *strag, real c, real *dinv);
template <typename real, typename st>
cudaError_t launch_energy_cn(const LaunchCtx &lc, const Dims &d, real *psi_k, const EnergyHalf<real, st> &h,
                             const GroupCoef<real> *coef, const StragCoef<real> *strag, const real *omega,
                             const real *dinv, double *flu_yz, double dose_scale, double flu_scale,
                             const BeamStrides &bs);

// The same with the explicit straggling term (strag != NULL), one lane per thread.
template <typename real, typename st>
cudaError_t launch_energy_strag(const LaunchCtx &lc, const Dims &d, real *psi_k, const EnergyHalf<real, st> &ha,
                                const EnergyHalf<real, st> *hb, const GroupCoef<real> *coef,
                                const StragCoef<real> *strag, double *flu_yz, double dose_scale, double flu_scale,
                                const BeamStrides &bs);

// The driver's tensor-map encoder (cuTensorMapEncodeTiled), looked up once
// through the runtime; NULL when the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

// Warp-per-plane streaming transport (k_transport_rows.cu).
template <typename real>
cudaError_t launch_transport_rows(const LaunchCtx &lc, const Dims &d, real *psi, double tau, double du, double dv,
                                  double dy, double dz);

template <typename real>
cudaError_t launch_angular(const LaunchCtx &lc, const Dims &d, real *psi, const real *rho_yz, const real *ts,
                           double h, double du, double dv);

bool angular_supported(int nu, int nv);
// Load the sine-transform tables into the current device's constant bank
// (synchronous; done once per context at creation).
cudaError_t angular_init_tables();

// src[b][g] = du dv P2_g R[b][g] for nbatch = n_beams source blocks of ng
// groups each (R, src laid out [b][g][a][yz]).
template <typename real, typename st>
cudaError_t launch_source(const LaunchCtx &lc, const Dims &d, const st *p2, const st *r, st *src, double dudv,
                          int nbatch = 1);

// R of one state for pbs_eval_source; precision as pbs_precision.
cudaError_t launch_source_input(const LaunchCtx &lc, const Dims &d, const void *psi_k, const void *rho_yz,
                                const void *coef, void *r_out, int precision);

// Persistent batch march (k_batch.cu).  One beam of the batch: its psi,
// density, tables, tallies, status word and the constants of its substeps
// (FP32), with the tile counts of its passes.
struct BatchBeam {
  float *psi;
  const float *rho;
  const GroupCoef<float> *coef;
  const float *ts;
  double *dose, *flu;
  int *err;
  Dims d;
  int n_steps;
  float c, hq, ky, kz, du, dv;  // E(h/2) CN factor, h/4 of A(h), transport tau/dy, tau/dz, angle spacings
  double dose_scale, flu_scale;
  int e_bx, a_bx, tr_kv, tr_nseg, tr_segw, tr_gw;
  long long tr_stacks;
};
// One task of the queue: pass `kind` of depth step `step` of a beam (for the
// transport and angular passes only the slab stacks first .. first+nstacks-1),
// split into ntiles tiles.  Its tiles start once counter wait_ctr has reached
// wait_need (wait_ctr < 0: at once) and each adds one to counter sig_ctr.
struct BatchTask {
  int beam, kind, step, wait_ctr, sig_ctr, pad;
  long long first, nstacks, ntiles, wait_need;
};
// Device counters of one launch (zeroed before it): the task being handed
// out and the abort word (per-beam completed tiles and per-task handed-out
// tiles are arrays of their own).
struct BatchQueue {
  unsigned long long cur;
  int abort, pad;
};
// Pass kinds of the batch queue.
namespace batch_pass {
enum : int { kPassEOpen = 0, kPassEPair = 1, kPassEClose = 2, kPassT = 3, kPassA = 4 };
}

// Tile counts and shared memory of one beam's passes in the batch kernel.
struct BatchShape {
  int e_bx, e_by;
  long long e_tiles, tr_stacks, t_tiles;
  int tr_kv, tr_nseg, tr_segw, tr_gw;
  int a_bx;
  long long a_tiles;
  size_t smem;
};
BatchShape batch_shape(const Dims &d, int shape, int cols);
bool batch_supported(int nu, int nv);
cudaError_t batch_init_tables();
// prof: NULL, or 8 counters the kernel adds to: SM clocks in energy,
// transport, angular tiles and in claiming/waiting ([0..3]) and the tiles
// run of each kind ([4..6]).  *ctas receives the launch's CTA count.
cudaError_t launch_batch(const LaunchCtx &lc, int shape, int nu, int nv, const BatchBeam *beams, int nbeams,
                         const BatchTask *tasks, int ntasks, BatchQueue *q, unsigned long long *done,
                         unsigned long long *next, long long wait_cycles, size_t smem, double du, double dv,
                         unsigned long long *prof, int *ctas);

template <typename real>
cudaError_t launch_init(const LaunchCtx &lc, const Dims &d, real *psi0, const double *fe, const double *fa,
                        const double *fy, const double *fz);

// Fluence of one beam: ncomp_beam components starting at psi.
template <typename real>
cudaError_t launch_fluence(const LaunchCtx &lc, const Dims &d, const real *psi, int ncomp_beam,
                           const GroupCoef<real> *coef, double *flu_yz, double scale);

}  // namespace pbs
