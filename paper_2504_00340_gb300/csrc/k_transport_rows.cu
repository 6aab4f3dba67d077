// k_transport_rows.cu -- lateral transport substep T(h) (Section 3.4, Eq.
// distansport, Remark 3), warp-per-plane streaming form.
//
// Flux-limited upwind finite volumes with the superbee slope, zero ghost
// cells, and the explicit trapezoid in depth  psi* = psi + h L(psi),  psi_new = (psi + psi* + h L(psi*))/2.
//
// GB300 design.  A group of lanes owns one (component, g, c, u, v) plane; each
// lane owns 4 adjacent z columns, so one row of up to 128 columns is one warp
// (wider rows are cut into segments with one halo lane per inner side).
//   * The scheme is symmetric under y -> -y and z -> -z, so each plane is
//     processed in a "march frame" in which both speeds are >= 0: rows are
//     visited from the last to the first when u < 0, and the lane -> column
//     map is mirrored when v < 0.  Every face flux is then the plain upwind
//     form  |s| (B + slope(B - A, C - B) / 2)  with no stencil selection, the
//     left edge is an inflow face (zero flux) and the flux through a lane's
//     left face is its left neighbour's right face (one shuffle).
//   * Rows arrive by per-lane cp.async (zero-filled out of range) into a
//     small per-warp ring in shared memory, kP rows ahead; a lane only reads
//     back what it copied, so no barrier is needed.
//   * Stage 1 (psi*) runs 1 row behind the newest row and stage 2 (psi_new)
//     2 rows behind, from sliding windows kept in registers; every face flux
//     is evaluated once per stage.
//   * psi_new is stored in place 2 rows behind the loads.
// Fluxes are pre-scaled by h/dy (h/dz): psi* = psi + (F_lo - F_hi) + (G_lo - G_hi).
#include "pbs_internal.cuh"
#include "transport_rows.cuh"

namespace pbs {

namespace {

using namespace tr;


constexpr int kWarps = 4;    // warps per CTA

template <typename real, bool VEC, bool FZ, int KV>
struct PlaneMarchCN : PlaneMarch<real, VEC, FZ, KV> {
  using B = PlaneMarch<real, VEC, FZ, KV>;
  using IO = typename B::IO;
  Vk<real, KV> xp;   // psi_new of the previous march row (zero before the first: inflow)
  real a, dinv, cy;  // sweep coefficients: a = cz / D, 1 / D, cy = h |u| / (2 dy)
  real apow[KV];     // a^(j+1)
  real aK;           // a^KV

  __device__ __forceinline__ void setup_cn() {
    cy = real(0.5) * this->sy;
    const real cz = real(0.5) * this->gz;
    dinv = real(1) / (real(1) + cy + cz);
    a = cz * dinv;
    real t = real(1);
#pragma unroll
    for (int j = 0; j < KV; j++) {
      t *= a;
      apow[j] = t;
    }
    aK = t;
#pragma unroll
    for (int j = 0; j < KV; j++) xp.v[j] = real(0);
  }

  // One iteration: LOAD row i; COMP: solve row m = i-1 (needs psi rows
  // m-2..m+1 = w[0..3]); FIRST: the first solved row (initialise the carried
  // y flux).
  template <bool LOAD, bool COMP, bool FIRST>
  __device__ __forceinline__ void iter_cn(int i) {
    Vk<real, KV> *w = this->w;
    cp_async_wait<kP - 1>();
    Vk<real, KV> x;
    if (LOAD) {
      IO::read(this->ring + this->rd * 32 * KV, x);
    } else {
#pragma unroll
      for (int j = 0; j < KV; j++) x.v[j] = real(0);
    }
    this->rd = (this->rd + 1) & (kR - 1);
    if (i + kP < this->ny) this->issue_row(this->ring + this->wr * 32 * KV, i + kP);
    cp_async_commit();
    this->wr = (this->wr + 1) & (kR - 1);
#pragma unroll
    for (int k = 0; k < 3; k++) w[k] = w[k + 1];
    w[3] = x;
    if (!COMP) return;
    const real sy = this->sy, gz = this->gz;
    if (FIRST) {
      const Vk<real, KV> d = sub4(w[2], w[1]);
      this->f1 = face4(sy, w[1], slope4(sub4(w[1], w[0]), d));
      this->e1 = d;
    }
    // psi + h L(psi): the limited operator on the old rows
    Vk<real, KV> dz;
    z_delta(w[2], gz, this->zl, this->zr, this->gw, dz);
    const Vk<real, KV> d = sub4(w[3], w[2]);
    const Vk<real, KV> fh = face4(sy, w[2], slope4(this->e1, d));
    this->e1 = d;
    const Vk<real, KV> s = upd4(w[2], this->f1, fh, dz);
    this->f1 = fh;
    // minus h/2 L1(psi), h L1 = sy (psi_{m-1} - psi_m) + gz (psi_{q-1} - psi_q)
    // (march frame: both speeds >= 0, zero ghosts upstream), then the
    // implicit upwind sweep  x_q = b_q + a x_{q-1},  b_q = (r_q + cy x_{m-1,q}) / D
    const real lft = this->zl * __shfl_up_sync(0xffffffffu, w[2].v[KV - 1], 1, this->gw);
    Vk<real, KV> y;
    real run = real(0);
#pragma unroll
    for (int j = 0; j < KV; j++) {
      const real zprev = j == 0 ? lft : w[2].v[j - 1];
      real r = s.v[j] - real(0.5) * (sy * (w[1].v[j] - w[2].v[j]) + gz * (zprev - w[2].v[j]));
      if (!VEC && this->col0 + j >= this->nz) r = real(0);
      const real b = (r + cy * xp.v[j]) * dinv;
      run = fma(a, run, b);
      y.v[j] = run;
    }
    // carry into the lane: x(first column - 1), a scan of the lanes' spans
    // x -> a^KV x + y_last over the lanes to the left (zero inflow at lane 0)
    real bsum = y.v[KV - 1], ad = aK;
    for (int dd = 1; dd < this->gw; dd <<= 1) {
      const real t = __shfl_up_sync(0xffffffffu, bsum, dd, this->gw);
      if (this->li >= dd) bsum = fma(ad, t, bsum);
      ad *= ad;
    }
    real xin = __shfl_up_sync(0xffffffffu, bsum, 1, this->gw);
    if (this->li == 0) xin = real(0);
#pragma unroll
    for (int j = 0; j < KV; j++) xp.v[j] = fma(apow[j], xin, y.v[j]);
    this->store_row(i - 1, xp);
  }

  __device__ __forceinline__ void run_cn() {
    this->prologue();
    setup_cn();
    const int ny = this->ny;
    iter_cn<true, false, false>(0);
    if (ny == 1) {
      iter_cn<false, true, true>(1);
      return;
    }
    iter_cn<true, true, true>(1);
#pragma unroll 4
    for (int i = 2; i < ny; i++) iter_cn<true, true, false>(i);
    iter_cn<false, true, false>(ny);
  }
};

template <typename real, bool VEC, bool FZ, int KV>
__device__ __forceinline__ void march_plane_cn(real *ring, real *pbase, int ny, int nz, int col0, int gw, int li,
                                               bool fwd, bool on, real sy, real gz, real zl, real zr) {
  PlaneMarchCN<real, VEC, FZ, KV> pm;
  pm.ring = ring;
  pm.pbase = pbase;
  pm.ny = ny;
  pm.nz = nz;
  pm.col0 = col0;
  pm.gw = gw;
  pm.li = li;
  pm.fwd = fwd;
  pm.on = on;
  pm.own = on;
  pm.sy = sy;
  pm.gz = gz;
  pm.zl = zl;
  pm.zr = zr;
  pm.run_cn();
}

// march_plane_cn as a function object for transport_tasks.
template <typename real, bool VEC, bool FZ, int KV>
struct MarchCn {
  __device__ __forceinline__ void operator()(real *ring, real *pbase, int ny, int nz, int col0, int gw, int li, bool fwd,
                                             bool on, real sy, real gz, real zl, real zr) const {
    march_plane_cn<real, VEC, FZ, KV>(ring, pbase, ny, nz, col0, gw, li, fwd, on, sy, gz, zl, zr);
  }
};

// Planes of one mirror class: FZ = the angles with v >= 0 (a >= a0, na_half
// of them per stack), else those with v < 0 (a < a0).  The two classes run as
// two launches so that each kernel holds one copy of the unrolled march.
//
// Rows wider than one warp's 32 lanes x 4 columns are cut into nseg segments
// of seg_w owned columns (march frame).  A segment's lane group also loads one
// lane of 4 columns on each inner side: the two Heun stages reach 4 columns
// upstream and 2 downstream, so the owned columns come out exact while the halo
// lanes' own results (their outer neighbours are missing) are discarded.  A
// task is one (plane, segment).
//
// CN: Crank-Nicolson with the slope lagged (Remark 3; see launch_transport_rows)
// instead of the explicit trapezoid; one segment per row.
// MINB > 1: registers capped so that MINB CTAs fit an SM (the 8-column
// march at three CTAs per SM).
template <typename real, bool VEC, bool FZ, int KV, bool CN, int MINB = 1>
__global__ void __launch_bounds__(kWarps * 32, MINB) k_transport_rows(real *__restrict__ psi, long long nplanes, int ny, int nz,
                                                                int na, int a0, int na_half, int nu, int nv, real du,
                                                                real dv, real ky, real kz, int nseg, int seg_w, int gw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  real *ring = reinterpret_cast<real *>(smem_raw) + (size_t)warp * kR * 32 * KV;
  transport_tasks<real, VEC, FZ, KV, CN>(psi, nplanes, ny, nz, na, a0, na_half, nu, nv, du, dv, ky, kz, nseg, seg_w, gw,
                                         lane, (long long)blockIdx.x * kWarps + warp, (long long)gridDim.x * kWarps,
                                         ring, MarchCn<real, VEC, FZ, KV>{});
}

// Segments of a row of nz columns: one if it fits a warp, else segments of at
// most 30 KV owned columns (with both halo lanes, 32 lanes).
void row_segments(int nz, int kv, int &nseg, int &seg_w, int &lanes) {
  if (nz <= 32 * kv) {
    nseg = 1;
    seg_w = nz;
    lanes = (nz + kv - 1) / kv;
    return;
  }
  const int wmax = (32 - 2) * kv;
  nseg = (nz + wmax - 1) / wmax;
  seg_w = ((nz + nseg - 1) / nseg + kv - 1) / kv * kv;
  lanes = seg_w / kv + 2;
}

// Fraction of the lane columns of the launched warps that hold owned columns.
double lane_use(int nz, int kv) {
  int nseg, seg_w, lanes;
  row_segments(nz, kv, nseg, seg_w, lanes);
  int gw = 1;
  while (gw < lanes) gw <<= 1;
  return (double)nz / ((double)nseg * gw * kv);
}

// Columns per lane: 6 where rows split evenly into 6-column lanes and that
// fills the warps better than 4 (rows of 48, 96 or 192 columns), else 4.
int pick_kv(int nz) {
  if (nz % 6 == 0 && lane_use(nz, 6) > lane_use(nz, 4) + 0.05) return 6;
  return 4;
}

template <typename real, int KV, bool CN>
cudaError_t launch_kv(const LaunchCtx &lc, const Dims &d, real *psi, double tau, double du, double dv, double dy,
                      double dz) {
  const long long nstacks = (long long)d.ncomp * d.ng * 2;
  // angles with v >= 0 (rows j >= nv / 2; for odd nv the middle row has v = 0)
  const int a_split = (d.nv / 2) * d.nu;
  int nseg, seg_w, lp;
  row_segments(d.nz, KV, nseg, seg_w, lp);
  int gw = 1;
  while (gw < lp) gw <<= 1;
  if (CN && nseg != 1) return cudaErrorNotSupported;  // the sweep runs along whole rows
  const bool vec = (d.nz % KV) == 0;
  const size_t smem = (size_t)kWarps * kR * 32 * KV * sizeof(real);
  for (int half = 0; half < 2; half++) {
    const bool fz = half == 1;
    const int a0 = fz ? a_split : 0;
    const int na_half = fz ? d.na - a_split : a_split;
    if (na_half == 0) continue;
    const long long nplanes = nstacks * na_half;
    auto kern = vec ? (fz ? k_transport_rows<real, true, true, KV, CN> : k_transport_rows<real, true, false, KV, CN>)
                    : (fz ? k_transport_rows<real, false, true, KV, CN> : k_transport_rows<real, false, false, KV, CN>);
    // the FP32 march needs a few registers more than some residencies leave
    // (4 columns: ~135, 8 columns: ~175): asked for 4 (4 columns) or 3 (8
    // columns) CTAs per SM, take the form whose registers are capped for it
    // (instantiated only for the FP32 explicit march: the other forms never
    // take them, and each capped pair is two more kernels to compile)
    if constexpr (sizeof(real) == 4 && !CN && (KV == 4 || KV == 8)) {
      constexpr int kCap = KV == 4 ? 4 : 3;
      if (vec && lc.transport_ctas == kCap)
        kern = fz ? k_transport_rows<real, true, true, KV, CN, kCap> : k_transport_rows<real, true, false, KV, CN, kCap>;
    }
    cudaError_t e;
    if (smem > 48 * 1024 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWarps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (lc.transport_ctas > 0 && lc.transport_ctas < per_sm) per_sm = lc.transport_ctas;
    const long long groups_per_block = (long long)kWarps * (32 / gw);
    long long blocks = (long long)per_sm * lc.num_sms;
    const long long need = (nplanes * nseg + groups_per_block - 1) / groups_per_block;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, kWarps * 32, smem, lc.stream>>>(psi, nplanes, d.ny, d.nz, d.na, a0, na_half, d.nu, d.nv,
                                                            (real)du, (real)dv, (real)(tau / dy), (real)(tau / dz), nseg,
                                                            seg_w, gw);
    ++*lc.launches;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

// Transport time integrator (Remark 3), lc.transport_cn:
//  0  explicit trapezoid (Heun) of the limited operator L;
//  1  Crank-Nicolson whose implicit half keeps the first-order upwind part
//     L1 implicit and takes the slope part from the old state:
//       (I - h/2 L1) psi_new = psi + h L(psi) - h/2 L1(psi),
//     one row at a time in the march frame: the right-hand side of row m
//     from the old rows m-2..m+1 (as stage 1 of Heun), then the implicit
//     part couples each cell to the new value upstream in y (the previous
//     row, in registers) and in z (its left neighbour): a first-order linear
//     recurrence along the row with the constant factor a = cz / D, run in
//     each lane over its columns and across lanes by a shuffle scan of the
//     lanes' affine maps (x -> a^KV x + y_last).  Rows of at most 32 KV
//     columns (one warp; 256 with KV = 8).
template <typename real>
cudaError_t launch_transport_rows(const LaunchCtx &lc, const Dims &d, real *psi, double tau, double du, double dv,
                                  double dy, double dz) {
  int kv = lc.transport_cols ? lc.transport_cols : pick_kv(d.nz);
  if (lc.transport_cn) {
    while (kv < 8 && d.nz > 32 * kv) kv = kv == 4 ? 6 : 8;  // the whole row in one warp
    if (d.nz > 32 * kv) return cudaErrorNotSupported;
    if (kv == 6) return launch_kv<real, 6, true>(lc, d, psi, tau, du, dv, dy, dz);
    if (kv == 8) return launch_kv<real, 8, true>(lc, d, psi, tau, du, dv, dy, dz);
    return launch_kv<real, 4, true>(lc, d, psi, tau, du, dv, dy, dz);
  }
  if (kv == 6) return launch_kv<real, 6, false>(lc, d, psi, tau, du, dv, dy, dz);
  if (kv == 8) return launch_kv<real, 8, false>(lc, d, psi, tau, du, dv, dy, dz);
  return launch_kv<real, 4, false>(lc, d, psi, tau, du, dv, dy, dz);
}

template cudaError_t launch_transport_rows<double>(const LaunchCtx &, const Dims &, double *, double, double, double,
                                                   double, double);
template cudaError_t launch_transport_rows<float>(const LaunchCtx &, const Dims &, float *, double, double, double,
                                                  double, double);

}  // namespace pbs
