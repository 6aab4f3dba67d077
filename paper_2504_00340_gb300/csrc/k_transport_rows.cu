// k_transport_rows.cu -- lateral transport substep T(h) (Section 3.4, Eq.
// distansport, Remark 3), warp-per-plane streaming form for nz <= 128.
//
// Same scheme as the tiled kernel in k_transport.cu: flux-limited upwind
// finite volumes with the superbee slope, zero ghost cells, and the explicit
// trapezoid in depth  psi* = psi + h L(psi),  psi_new = (psi + psi* + h L(psi*))/2.
//
// GB300 design.  A group of lanes owns one (component, g, c, u, v) plane; each
// lane owns 4 adjacent z columns, so one row of up to 128 columns is one warp.
// The group streams down the plane one row per iteration:
//   * rows arrive by per-lane cp.async (16-byte, zero-filled out of range)
//     into a small per-warp ring in shared memory, P rows ahead; a lane only
//     reads back what it copied, so no barrier is needed;
//   * in the march frame the flow is positive, so a face flux only looks
//     upstream: stage 1 (psi*) runs 1 row behind the newest row and stage 2
//     (psi_new) 2 rows behind, both from sliding windows of 4 rows kept in
//     registers; every y face flux is evaluated once;
//   * z neighbours across lanes come from warp shuffles;
//   * when u < 0 the group marches from the last row to the first, so in the
//     march frame the y flow is always positive and the upwind stencil needs
//     no selection (the scheme is symmetric under y -> -y);
//   * psi_new is stored in place 2 rows behind the loads.
// Fluxes are pre-scaled by h/dy (h/dz), so psi* = psi + (F_lo - F_hi) + (G_lo - G_hi).
#include "pbs_internal.cuh"

namespace pbs {

namespace {

constexpr int kV = 4;        // columns per lane
constexpr int kP = 6;        // rows in flight per lane
constexpr int kR = kP + 1;   // ring slots
constexpr int kWarps = 4;    // warps per CTA

template <typename real>
struct V4 {
  real v[kV];
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, unsigned src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Upwind face value for flow from A through B to C (positive direction):
//   B + slope(B - A, C - B) / 2, with the superbee slope.
template <typename real>
__device__ __forceinline__ real face_value(real A, real B, real C) {
  const real d1 = B - A, d2 = C - B;
  const real a1 = fabs(d1), a2 = fabs(d2);
  const real m = fmin(fmax(a1, a2), real(2) * fmin(a1, a2));  // zero if either difference is zero
  const real sl = same_sign(d1, d2) ? copysign(m, d2) : real(0);
  return fma(real(0.5), sl, B);
}

template <typename real, bool VEC>
struct RowIO {
  // Issue the copy of row `row` (columns col0..col0+3) of a plane into `dst`.
  static __device__ __forceinline__ void issue(real *dst, const real *plane_base, int row, int nz, int col0, bool on) {
    const real *src = plane_base + (long long)row * nz + col0;
    if (VEC) {
      const unsigned nb = on ? 16u : 0u;
#pragma unroll
      for (int k = 0; k < (int)(kV * sizeof(real) / 16); k++)
        cp_async16(dst + k * (16 / sizeof(real)), on ? src + k * (16 / sizeof(real)) : plane_base, nb);
    } else {
#pragma unroll
      for (int k = 0; k < kV; k++) {
        const bool in = on && (col0 + k < nz);
        if (sizeof(real) == 8)
          cp_async8(dst + k, in ? src + k : plane_base, in ? 8u : 0u);
        else
          cp_async4(dst + k, in ? src + k : plane_base, in ? 4u : 0u);
      }
    }
  }
  static __device__ __forceinline__ void store(real *plane_base, int row, int nz, int col0, bool on, const V4<real> &x) {
    if (!on) return;
    real *dst = plane_base + (long long)row * nz + col0;
    if (VEC) {
      if (sizeof(real) == 4) {
        *reinterpret_cast<float4 *>(dst) = make_float4((float)x.v[0], (float)x.v[1], (float)x.v[2], (float)x.v[3]);
      } else {
        reinterpret_cast<double2 *>(dst)[0] = make_double2((double)x.v[0], (double)x.v[1]);
        reinterpret_cast<double2 *>(dst)[1] = make_double2((double)x.v[2], (double)x.v[3]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < kV; k++)
        if (col0 + k < nz) dst[k] = x.v[k];
    }
  }
};

// z-direction contribution G_lo - G_hi for the lane's 4 cells of one row.
// gs: signed v * h / dz.  Neighbour columns come from the adjacent lanes of
// the group (zero at the plane's edges).
template <typename real>
__device__ __forceinline__ void z_delta(const V4<real> &c, real gs, bool vpos, int li, int lp, int gw, V4<real> &out) {
  real l2 = __shfl_up_sync(0xffffffffu, c.v[2], 1, gw);
  real l1 = __shfl_up_sync(0xffffffffu, c.v[3], 1, gw);
  real r1 = __shfl_down_sync(0xffffffffu, c.v[0], 1, gw);
  real r2 = __shfl_down_sync(0xffffffffu, c.v[1], 1, gw);
  if (li == 0) { l2 = real(0); l1 = real(0); }
  if (li >= lp - 1) { r1 = real(0); r2 = real(0); }
  const real x[8] = {l2, l1, c.v[0], c.v[1], c.v[2], c.v[3], r1, r2};
  real g[5];
#pragma unroll
  for (int k = 0; k < 5; k++) {
    // face between x[k+1] and x[k+2]
    const real A = vpos ? x[k] : x[k + 3];
    const real B = vpos ? x[k + 1] : x[k + 2];
    const real C = vpos ? x[k + 2] : x[k + 1];
    g[k] = gs * face_value(A, B, C);
  }
#pragma unroll
  for (int j = 0; j < kV; j++) out.v[j] = g[j] - g[j + 1];
}

template <typename real, bool VEC>
__global__ void __launch_bounds__(kWarps * 32) k_transport_rows(real *__restrict__ psi, long long nplanes, int ny, int nz,
                                                                int na, int nu, int nv, real du, real dv, real ky,
                                                                real kz, int lp, int gw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  real *ring = reinterpret_cast<real *>(smem_raw) + ((size_t)warp * kR * 32 + lane) * kV;  // slot stride 32*kV
  const int ngroups = 32 / gw;
  const int gi = lane / gw;
  const int li = lane % gw;
  const int col0 = li * kV;
  const bool lane_on = li < lp;
  const long long gwarp = (long long)blockIdx.x * kWarps + warp;
  const long long nwarps = (long long)gridDim.x * kWarps;

  for (long long base = gwarp * ngroups; base < nplanes; base += nwarps * ngroups) {
    const long long plane = base + gi;
    const bool valid = plane < nplanes;
    const bool on = valid && lane_on;
    const int a = valid ? (int)(plane % na) : 0;
    const real uu = (real)((a % nu) - 0.5 * (nu - 1)) * du;
    const real vv = (real)((a / nu) - 0.5 * (nv - 1)) * dv;
    const bool fwd = uu >= real(0);
    const real sy = fabs(uu) * ky;  // |u| h / dy in the march frame
    const real gz = vv * kz;        // v h / dz (signed)
    const bool vpos = vv > real(0);
    real *pbase = psi + (valid ? plane : 0) * (long long)ny * nz;

    // prologue: rows 0..kP-1 of the march order
    int wr = 0;
#pragma unroll
    for (int j = 0; j < kP; j++) {
      if (j < ny) RowIO<real, VEC>::issue(ring + wr * 32 * kV, pbase, fwd ? j : ny - 1 - j, nz, col0, on);
      cp_async_commit();
      wr++;
    }
    int rd = 0;
    // w: psi of march rows i-3..i; st: psi* of march rows i-4..i-1
    V4<real> w[4], st[4];
#pragma unroll
    for (int k = 0; k < 4; k++)
#pragma unroll
      for (int j = 0; j < kV; j++) w[k].v[j] = st[k].v[j] = real(0);
    V4<real> f1, f2;  // carried y face fluxes (face m - 1/2) of stage 1 and stage 2
#pragma unroll
    for (int j = 0; j < kV; j++) f1.v[j] = f2.v[j] = real(0);

    for (int i = 0; i < ny + 2; i++) {
      cp_async_wait<kP - 1>();
      V4<real> x;
      if (i < ny) {
        const real *src = ring + rd * 32 * kV;
#pragma unroll
        for (int j = 0; j < kV; j++) x.v[j] = src[j];
      } else {
#pragma unroll
        for (int j = 0; j < kV; j++) x.v[j] = real(0);
      }
      rd = (rd + 1 == kR) ? 0 : rd + 1;
      if (i + kP < ny) RowIO<real, VEC>::issue(ring + wr * 32 * kV, pbase, fwd ? i + kP : ny - 1 - (i + kP), nz, col0, on);
      cp_async_commit();
      wr = (wr + 1 == kR) ? 0 : wr + 1;
#pragma unroll
      for (int k = 0; k < 3; k++) w[k] = w[k + 1];
      w[3] = x;

      if (i >= 1) {  // stage 1 for march row m = i-1: needs psi(m-2..m+1) = w[0..3]
        if (i == 1) {
#pragma unroll
          for (int j = 0; j < kV; j++) f1.v[j] = sy * face_value(w[0].v[j], w[1].v[j], w[2].v[j]);
        }
        V4<real> dz, s;
        z_delta(w[2], gz, vpos, li, lp, gw, dz);
        const bool row_in = (i - 1) < ny;
#pragma unroll
        for (int j = 0; j < kV; j++) {
          const real fh = sy * face_value(w[1].v[j], w[2].v[j], w[3].v[j]);  // face m + 1/2
          s.v[j] = (row_in && col0 + j < nz) ? w[2].v[j] + (f1.v[j] - fh) + dz.v[j] : real(0);
          f1.v[j] = fh;
        }
#pragma unroll
        for (int k = 0; k < 3; k++) st[k] = st[k + 1];
        st[3] = s;
      }
      if (i >= 2) {  // stage 2 for march row m' = i-2: needs psi*(m'-2..m'+1) = st[0..3], psi(m') = w[1]
        if (i == 2) {
#pragma unroll
          for (int j = 0; j < kV; j++) f2.v[j] = sy * face_value(st[0].v[j], st[1].v[j], st[2].v[j]);
        }
        V4<real> dz, o;
        z_delta(st[2], gz, vpos, li, lp, gw, dz);
#pragma unroll
        for (int j = 0; j < kV; j++) {
          const real fh = sy * face_value(st[1].v[j], st[2].v[j], st[3].v[j]);
          o.v[j] = real(0.5) * (w[1].v[j] + st[2].v[j] + (f2.v[j] - fh) + dz.v[j]);
          f2.v[j] = fh;
        }
        const int r2 = i - 2;
        RowIO<real, VEC>::store(pbase, fwd ? r2 : ny - 1 - r2, nz, col0, on, o);
      }
    }
  }
  cp_async_wait<0>();
}

}  // namespace

bool transport_rows_supported(int nz) { return nz >= 1 && nz <= 32 * kV; }

template <typename real>
cudaError_t launch_transport_rows(const LaunchCtx &lc, const Dims &d, real *psi, double tau, double du, double dv,
                                  double dy, double dz) {
  const long long nplanes = (long long)d.ncomp * d.ng * 2 * d.na;
  const int lp = (d.nz + kV - 1) / kV;
  int gw = 1;
  while (gw < lp) gw <<= 1;
  const bool vec = (d.nz % kV) == 0;
  const size_t smem = (size_t)kWarps * kR * 32 * kV * sizeof(real);
  auto kern = vec ? k_transport_rows<real, true> : k_transport_rows<real, false>;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long groups_per_block = (long long)kWarps * (32 / gw);
  long long blocks = (long long)per_sm * lc.num_sms;
  const long long need = (nplanes + groups_per_block - 1) / groups_per_block;
  if (blocks > need) blocks = need;
  kern<<<(unsigned)blocks, kWarps * 32, smem, lc.stream>>>(psi, nplanes, d.ny, d.nz, d.na, d.nu, d.nv, (real)du,
                                                          (real)dv, (real)(tau / dy), (real)(tau / dz), lp, gw);
  ++*lc.launches;
  return cudaGetLastError();
}

template cudaError_t launch_transport_rows<double>(const LaunchCtx &, const Dims &, double *, double, double, double,
                                                   double, double);
template cudaError_t launch_transport_rows<float>(const LaunchCtx &, const Dims &, float *, double, double, double,
                                                  double, double);

}  // namespace pbs
