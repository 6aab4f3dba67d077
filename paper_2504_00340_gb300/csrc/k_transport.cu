// k_transport.cu -- lateral transport substep T(h) (Section 3.4, Eq.
// distansport, Remark 3): flux-limited upwind finite volumes in (y, z) at the
// plane's angle (u_i, v_j), zero ghost cells, superbee slope, and the explicit
// trapezoid (Heun) in depth that Remark 3's explicit slope treatment gives:
//   psi* = psi + h L(psi),   psi_new = (psi + psi* + h L(psi*)) / 2.
//
// GB300 design.  Every (component, g, c, u, v) plane is an Ny x Nz block of
// contiguous memory.  A persistent CTA owns whole planes and streams down
// each one in chunks of TY rows:
//   * chunk rows arrive by 1-D TMA bulk copies (cp.async.bulk) into a ring of
//     kSlots chunk buffers in shared memory, issued kSlots-1 chunks ahead and
//     tracked by one mbarrier per slot (bounded waits);
//   * stage 1 computes psi* for rows [y0+2, y0+TY+2) (rows 0.. for the first
//     chunk) into a ring of 2*TY rows; rows y0-2..y0+1 were made by the
//     previous chunk, so no halo row is loaded or recomputed twice;
//   * stage 2 writes psi_new for rows [y0, y0+TY) straight to global memory.
// Each thread owns one column z and a contiguous run of rows, so the y face
// fluxes slide down the run (one flux evaluation per face); the z neighbours
// come from the shared-memory row.  Because a CTA finishes a plane's chunks in
// order and keeps the old halo rows in shared memory, the update is in place.
#include "pbs_internal.cuh"

namespace pbs {

namespace {

constexpr int kSlots = 4;
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

struct TransportShape {
  int ny, nz, ty, nchunk, rseg;  // rseg: row segments per chunk (threads = nz * rseg)
  long long nplanes;
  int na, nu;
};

template <typename real>
__global__ void k_transport(TransportShape sh, real *__restrict__ psi, real tau, real inv_dy, real inv_dz,
                            real du, real dv, int nv, int bulk_ok, int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int ny = sh.ny, nz = sh.nz, TY = sh.ty;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
  real *ring = reinterpret_cast<real *>(smem_raw + 128);   // kSlots * TY * nz
  real *star = ring + (size_t)kSlots * TY * nz;             // 2 * TY * nz
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int q = tid % nz;
  const int seg = tid / nz;
  const long long nitems_per_plane = sh.nchunk;
  // planes owned by this CTA: blockIdx.x, blockIdx.x + gridDim.x, ...
  const long long my_planes =
      (sh.nplanes > blockIdx.x) ? (sh.nplanes - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long nitems = my_planes * nitems_per_plane;

  if (tid == 0) {
    for (int s = 0; s < kSlots; s++) mbar_init(&bars[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();

  auto item_plane = [&](long long i) -> long long { return blockIdx.x + (i / nitems_per_plane) * gridDim.x; };
  auto item_chunk = [&](long long i) -> int { return (int)(i % nitems_per_plane); };

  // Issue the load of item i into slot i % kSlots (called by all threads).
  auto issue = [&](long long i) {
    if (i >= nitems) return;
    const long long plane = item_plane(i);
    const int ch = item_chunk(i);
    const int r0 = ch * TY;
    const int rows = min(TY, ny - r0);
    real *dst = ring + (size_t)(i % kSlots) * TY * nz;
    const real *src = psi + (plane * ny + r0) * (long long)nz;
    if (bulk_ok) {
      if (tid == 0) {
        fence_proxy_async_smem();
        const unsigned bytes = (unsigned)(rows * nz * sizeof(real));
        mbar_arrive_expect_tx(&bars[i % kSlots], bytes);
        bulk_g2s(dst, src, bytes, &bars[i % kSlots]);
      }
    } else {
      for (int e = tid; e < rows * nz; e += blockDim.x) dst[e] = src[e];
    }
  };
  // Make item i's rows visible (bounded wait); returns false on timeout.
  auto ready = [&](long long i) -> bool {
    if (i >= nitems || !bulk_ok) return true;
    if (tid == 0) {
      if (!mbar_wait_bounded(&bars[i % kSlots], (unsigned)((i / kSlots) & 1), kWaitCycles)) s_abort = 1;
    }
    return true;
  };

  for (int i = 0; i < kSlots - 1; i++) issue(i);
  long long issued = kSlots - 1;  // items [0, issued) have been issued
  long long it = 0;

  for (; it < nitems; it++) {
    issue(it + kSlots - 1);  // its slot held item it-1, finished at the last barrier
    issued = it + kSlots;
    const long long plane = item_plane(it);
    const int ch = item_chunk(it);
    const int y0 = ch * TY;
    const bool has_next = (ch + 1 < sh.nchunk);
    ready(it);
    if (has_next) ready(it + 1);
    __syncthreads();
    if (s_abort) break;

    const int a = (int)(plane % sh.na);
    const real uu = (real)((a % sh.nu) - 0.5 * (sh.nu - 1)) * du;
    const real vv = (real)((a / sh.nu) - 0.5 * (nv - 1)) * dv;
    const bool upos = uu > real(0), vpos = vv > real(0);

    // psi at (row r, column cc) for rows r in [y0-4, y0+TY+4); zero outside the grid
    const real *slot0 = ring + (size_t)(it % kSlots) * TY * nz;
    const real *slot1 = ring + (size_t)((it + 1) % kSlots) * TY * nz;
    auto P = [&](int r, int cc) -> real {
      if (r < 0 || r >= ny || cc < 0 || cc >= nz) return real(0);
      const int off = r - y0;
      return off < TY ? slot0[off * nz + cc] : slot1[(off - TY) * nz + cc];
    };
    auto S = [&](int r, int cc) -> real {
      if (r < 0 || r >= ny || cc < 0 || cc >= nz) return real(0);
      return star[(size_t)(r % (2 * TY)) * nz + cc];
    };

    // ---- stage 1: psi* rows [s_lo, s_hi)
    {
      const int s_lo = (ch == 0) ? 0 : y0 + 2;
      const int s_hi = min(ny, y0 + TY + 2);
      const int n = s_hi - s_lo;
      if (n > 0 && seg < sh.rseg) {
        const int per = (n + sh.rseg - 1) / sh.rseg;
        const int r_beg = s_lo + seg * per;
        const int r_end = min(s_hi, r_beg + per);
        if (r_beg < r_end) {
          real w0 = P(r_beg - 2, q), w1 = P(r_beg - 1, q), w2 = P(r_beg, q), w3 = P(r_beg + 1, q);
          real w4 = P(r_beg + 2, q);
          real f_lo = face_flux(upos, uu, w0, w1, w2, w3);
          for (int r = r_beg; r < r_end; r++) {
            const real f_hi = face_flux(upos, uu, w1, w2, w3, w4);
            const real zm2 = P(r, q - 2), zm1 = P(r, q - 1), zp1 = P(r, q + 1), zp2 = P(r, q + 2);
            const real g_lo = face_flux(vpos, vv, zm2, zm1, w2, zp1);
            const real g_hi = face_flux(vpos, vv, zm1, w2, zp1, zp2);
            const real l0 = -(f_hi - f_lo) * inv_dy - (g_hi - g_lo) * inv_dz;
            star[(size_t)(r % (2 * TY)) * nz + q] = w2 + tau * l0;
            f_lo = f_hi;
            w0 = w1; w1 = w2; w2 = w3; w3 = w4;
            if (r + 1 < r_end) w4 = P(r + 3, q);
          }
        }
      }
    }
    __syncthreads();
    // ---- stage 2: psi_new rows [y0, y0+TY)
    {
      const int r_hi = min(ny, y0 + TY);
      const int n = r_hi - y0;
      if (seg < sh.rseg) {
        const int per = (n + sh.rseg - 1) / sh.rseg;
        const int r_beg = y0 + seg * per;
        const int r_end = min(r_hi, r_beg + per);
        if (r_beg < r_end) {
          real w0 = S(r_beg - 2, q), w1 = S(r_beg - 1, q), w2 = S(r_beg, q), w3 = S(r_beg + 1, q);
          real w4 = S(r_beg + 2, q);
          real f_lo = face_flux(upos, uu, w0, w1, w2, w3);
          real *out = psi + (plane * ny) * (long long)nz + q;
          for (int r = r_beg; r < r_end; r++) {
            const real f_hi = face_flux(upos, uu, w1, w2, w3, w4);
            const real zm2 = S(r, q - 2), zm1 = S(r, q - 1), zp1 = S(r, q + 1), zp2 = S(r, q + 2);
            const real g_lo = face_flux(vpos, vv, zm2, zm1, w2, zp1);
            const real g_hi = face_flux(vpos, vv, zm1, w2, zp1, zp2);
            const real l1 = -(f_hi - f_lo) * inv_dy - (g_hi - g_lo) * inv_dz;
            out[(long long)r * nz] = real(0.5) * (P(r, q) + w2 + tau * l1);
            f_lo = f_hi;
            w0 = w1; w1 = w2; w2 = w3; w3 = w4;
            if (r + 1 < r_end) w4 = S(r + 3, q);
          }
        }
      }
    }
    __syncthreads();
  }
  if (s_abort && tid == 0) {
    atomicAdd(err, 1);
    atomicExch(err + 1, kErrTimeoutTransport);
    // let the copies still in flight land before this CTA's shared memory is
    // released (bounded as well)
    if (bulk_ok) {
      const long long last = issued < nitems ? issued : nitems;
      for (long long j = it; j < last; j++)
        mbar_wait_bounded(&bars[j % kSlots], (unsigned)((j / kSlots) & 1), kWaitCycles / 8);
    }
  }
}

}  // namespace

template <typename real>
cudaError_t launch_transport(const LaunchCtx &lc, const Dims &d, real *psi, double tau, double du, double dv,
                             double dy, double dz, int *err) {
  TransportShape sh;
  sh.ny = d.ny;
  sh.nz = d.nz;
  sh.na = d.na;
  sh.nu = d.nu;
  sh.nplanes = (long long)d.ncomp * d.ng * 2 * d.na;
  // chunk height: 16 rows (8 for wide FP64 rows) and at least 4 (halo)
  int ty = (d.nz * (int)sizeof(real) > 1024) ? 8 : 16;
  if (ty > d.ny) ty = d.ny < 4 ? 4 : d.ny;
  sh.ty = ty;
  sh.nchunk = (d.ny + ty - 1) / ty;
  int rseg = 256 / d.nz;
  if (rseg < 1) rseg = 1;
  if (rseg > ty) rseg = ty;
  sh.rseg = rseg;
  const int threads = d.nz * rseg;
  const size_t smem = 128 + (size_t)(kSlots * ty + 2 * ty) * d.nz * sizeof(real);
  const int bulk_ok = ((d.nz * sizeof(real)) % 16 == 0) ? 1 : 0;
  cudaError_t e = cudaFuncSetAttribute(k_transport<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transport<real>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long blocks = (long long)per_sm * lc.num_sms;
  if (blocks > sh.nplanes) blocks = sh.nplanes;
  k_transport<real><<<(unsigned)blocks, threads, smem, lc.stream>>>(
      sh, psi, (real)tau, (real)(1.0 / dy), (real)(1.0 / dz), (real)du, (real)dv, d.nv, bulk_ok, err);
  ++*lc.launches;
  return cudaGetLastError();
}

template cudaError_t launch_transport<double>(const LaunchCtx &, const Dims &, double *, double, double, double,
                                              double, double, int *);
template cudaError_t launch_transport<float>(const LaunchCtx &, const Dims &, float *, double, double, double,
                                             double, double, int *);

}  // namespace pbs
