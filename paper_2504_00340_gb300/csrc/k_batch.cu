// k_batch.cu -- the depth march of a whole batch of pencil beams (spots) in
// one persistent launch.
//
// Each beam is its own context (own grid, energy groups, tables, density and
// workspace).  Its march is a chain of passes over its psi: per depth step s
// the Strang sequence of Section 3.3 as four passes,
//   E(h/2) [closing step s-1, fused with opening step s]   T(h/2)   A(h)   T(h/2),
// and after its last step the closing E(h/2).  Each pass splits into tiles:
// the blocks of the per-substep kernels (the same device code, energy_f2.cuh,
// transport_rows.cuh, angular_f2.cuh), so a tile computes exactly what the
// corresponding block of the ordinary launch computes.
//
// The queue is a host-built list of (beam, pass) tasks, round-robin over the
// beams (pass 0 of every beam, then pass 1 of every beam still marching, ...).
// The CTAs of one persistent launch hand out the tiles of the current task
// through its counter and advance the task index when it runs dry, so tiles
// leave the queue in task order.  A tile of pass p of beam b waits until b's
// completion counter has reached the number of b's tiles in passes before p;
// every tile it waits for left the queue earlier, to a CTA that is running
// and whose own wait is on still earlier tiles, so the waits always end.
// Each wait is bounded (SM clocks): a wait that gives up sets the batch abort
// word and every beam's device status word, and every CTA stops at its next
// tile boundary, with nothing in flight.
#include "pbs_internal.cuh"
#include "angular_f2.cuh"
#include "energy_f2.cuh"
#include "transport_rows.cuh"

#include <algorithm>

namespace pbs {

namespace {

constexpr int kBThreads = 128;  // the energy block (32 x 4), the angular block (16 x 8), four transport warps
constexpr int kBWarps = kBThreads / 32;
constexpr int kBKV = 4;         // transport columns per lane
constexpr int kBEnergyY = 4;    // energy block rows: 8 angles per block
constexpr int kBAngRep = 16;    // angular slab stacks per tile

// Pass kinds of a beam's chain.
enum : int { kPassEOpen = 0, kPassEPair = 1, kPassEClose = 2, kPassT = 3, kPassA = 4 };

__device__ __forceinline__ int pass_kind(int pass, int n_steps) {
  if (pass == 4 * n_steps) return kPassEClose;
  switch (pass & 3) {
    case 0: return pass == 0 ? kPassEOpen : kPassEPair;
    case 2: return kPassA;
    default: return kPassT;
  }
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_i(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Give up the whole batch: the abort word, and every beam's status word.
__device__ void batch_abort(const BatchBeam *beams, int nbeams, int *abort_word, int where) {
  if (atomicCAS(abort_word, 0, where) == 0) {
    for (int b = 0; b < nbeams; b++) {
      if (beams[b].err) {
        atomicAdd(beams[b].err, 1);
        atomicExch(beams[b].err + 1, kErrTimeoutBatch);
      }
    }
  }
}

template <int NU, int NV>
__device__ __forceinline__ void run_tile(const BatchBeam &bm, int kind, int step, long long tile, unsigned char *smem,
                                         const ang::AngTables<float> &tb) {
  const Dims &d = bm.d;
  const int tid = threadIdx.x;
  const size_t nyz = (size_t)d.nyz;
  if (kind == kPassEOpen || kind == kPassEPair || kind == kPassEClose) {
    const int bx = (int)(tile % bm.e_bx), by = (int)(tile / bm.e_bx);
    const BeamStrides bs{0, 0, 0, 0};
    // E(h/2) with the density of slab sa: opening step 0, closing the last
    // step, or closing step - 1 fused with opening step (its slab), with the
    // fluence after the closing half
    const int sa = kind == kPassEOpen ? 0 : step - 1;
    if (kind == kPassEPair) {
      en::energy_f2_tile<float, false, false, true, kBEnergyY>(
          bx, by, 0, tid & 31, tid >> 5, smem, d, bm.psi, nullptr, nullptr, nullptr, nullptr, bm.rho + sa * nyz,
          bm.rho + (size_t)step * nyz, bm.coef, bm.dose + sa * nyz, bm.dose + (size_t)step * nyz,
          bm.flu + (size_t)step * nyz, bm.c, bm.c, bm.dose_scale, bm.flu_scale, bs);
    } else {
      double *flu = kind == kPassEClose ? bm.flu + (size_t)bm.n_steps * nyz : nullptr;
      en::energy_f2_tile<float, false, false, false, kBEnergyY>(
          bx, by, 0, tid & 31, tid >> 5, smem, d, bm.psi, nullptr, nullptr, nullptr, nullptr, bm.rho + sa * nyz,
          nullptr, bm.coef, bm.dose + sa * nyz, nullptr, flu, bm.c, bm.c, bm.dose_scale, bm.flu_scale, bs);
    }
  } else if (kind == kPassT) {
    // one slab stack (component, g, c) of one mirror class per tile
    const long long nst = bm.tr_stacks;
    const int fz = tile >= nst ? 1 : 0;
    const long long stack = fz ? tile - nst : tile;
    const int a_split = (d.nv / 2) * d.nu;
    const int a0 = fz ? a_split : 0, na_half = fz ? d.na - a_split : a_split;
    float *psi = bm.psi + stack * (long long)d.na * d.nyz;
    const int lane = tid & 31, warp = tid >> 5;
    float *ring = reinterpret_cast<float *>(smem) + (size_t)warp * tr::kR * 32 * kBKV;
    if (fz)
      tr::transport_tasks<float, true, true, kBKV, false>(psi, na_half, d.ny, d.nz, d.na, a0, na_half, d.nu, d.nv,
                                                          bm.du, bm.dv, bm.ky, bm.kz, bm.tr_nseg, bm.tr_segw,
                                                          bm.tr_gw, lane, warp, kBWarps, ring, tr::NoCnMarch{});
    else
      tr::transport_tasks<float, true, false, kBKV, false>(psi, na_half, d.ny, d.nz, d.na, a0, na_half, d.nu, d.nv,
                                                           bm.du, bm.dv, bm.ky, bm.kz, bm.tr_nseg, bm.tr_segw,
                                                           bm.tr_gw, lane, warp, kBWarps, ring, tr::NoCnMarch{});
  } else {  // kPassA: kBAngRep consecutive slab stacks at one lateral block
    const int bx = (int)(tile % bm.a_bx);
    const long long k0 = (tile / bm.a_bx) * kBAngRep;
    const long long nkgc = (long long)d.ncomp * d.ng * 2;
    for (int r = 0; r < kBAngRep && k0 + r < nkgc; r++) {
      ang::angular_f2_tile<NU, NV, false>(bm.psi, bm.rho + (size_t)step * nyz, bm.ts, d.nyz, d.ng, bm.hq, k0 + r, bx,
                                         tid & 15, tid >> 4, smem, tb);
      __syncthreads();  // the next stack reuses the shared tile
    }
  }
}

template <int NU, int NV>
__global__ void __launch_bounds__(kBThreads, 4)
    k_batch(const BatchBeam *__restrict__ beams, int nbeams, const BatchTask *__restrict__ tasks, int ntasks,
            BatchQueue *q, unsigned long long *done_ctr, unsigned long long *next_ctr, long long wait_cycles,
            const __grid_constant__ ang::AngTables<float> tb) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_task, s_go;
  __shared__ long long s_tile;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      int go = 0, t = 0;
      long long tile = 0;
      for (;;) {
        if (ld_acquire_i(&q->abort) != 0) break;
        t = (int)ld_acquire(&q->cur);
        if (t >= ntasks) break;
        tile = (long long)atomicAdd(&next_ctr[t], 1ULL);
        if (tile < tasks[t].ntiles) {
          go = 1;
          break;
        }
        atomicCAS(&q->cur, (unsigned long long)t, (unsigned long long)t + 1);  // this task is handed out
      }
      if (go) {
        // the beam's earlier passes: every one of their tiles has completed
        const BatchTask tk = tasks[t];
        const unsigned long long need = (unsigned long long)tk.need;
        unsigned long long *done = &done_ctr[tk.beam];
        if (ld_acquire(done) < need) {
          const long long t0 = clock64();
          while (ld_acquire(done) < need) {
            if (ld_acquire_i(&q->abort) != 0) {
              go = 0;
              break;
            }
            if (clock64() - t0 > wait_cycles) {
              batch_abort(beams, nbeams, &q->abort, 1 + tk.beam);
              go = 0;
              break;
            }
            __nanosleep(200);
          }
        }
      }
      s_task = t;
      s_tile = tile;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) break;
    const BatchTask tk = tasks[s_task];
    const BatchBeam &bm = beams[tk.beam];
    run_tile<NU, NV>(bm, pass_kind(tk.pass, bm.n_steps), tk.pass >> 2, s_tile, smem, tb);
    __syncthreads();  // every thread's writes of this tile are done
    if (tid == 0) {
      __threadfence();
      atomicAdd(&done_ctr[tk.beam], 1ULL);
    }
  }
}

template <int NU, int NV>
cudaError_t go_batch(const LaunchCtx &lc, const BatchBeam *beams, int nbeams, const BatchTask *tasks, int ntasks,
                     BatchQueue *q, unsigned long long *done, unsigned long long *next, long long wait_cycles,
                     size_t smem, double du, double dv) {
  auto kern = k_batch<NU, NV>;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBThreads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  ang::AngTables<float> tb;
  ang::fill_tables(tb, NU, NV, du, dv);
  // A CTA only ever waits for tiles that left the queue before its own, that
  // is, for tiles held by CTAs already running: the launch needs no
  // co-residency guarantee (and so stays capturable in a graph).
  kern<<<(unsigned)(per_sm * lc.num_sms), kBThreads, smem, lc.stream>>>(beams, nbeams, tasks, ntasks, q, done, next,
                                                                        wait_cycles, tb);
  ++*lc.launches;
  return cudaGetLastError();
}

}  // namespace

cudaError_t batch_init_tables() { return ang::upload_dst_f2(); }

BatchShape batch_shape(const Dims &d) {
  BatchShape s{};
  s.e_bx = (d.nyz / 2 + en::kX - 1) / en::kX;
  s.e_by = (d.na + kBEnergyY * en::kA - 1) / (kBEnergyY * en::kA);
  s.e_tiles = (long long)s.e_bx * s.e_by;
  s.tr_stacks = (long long)d.ncomp * d.ng * 2;
  s.t_tiles = 2 * s.tr_stacks;
  int nseg, seg_w, lanes;
  nseg = 1;
  seg_w = d.nz;
  lanes = (d.nz + kBKV - 1) / kBKV;
  if (d.nz > 32 * kBKV) {  // rows cut into segments as in the per-substep kernel
    const int wmax = (32 - 2) * kBKV;
    nseg = (d.nz + wmax - 1) / wmax;
    seg_w = ((d.nz + nseg - 1) / nseg + kBKV - 1) / kBKV * kBKV;
    lanes = seg_w / kBKV + 2;
  }
  int gw = 1;
  while (gw < lanes) gw <<= 1;
  s.tr_nseg = nseg;
  s.tr_segw = seg_w;
  s.tr_gw = gw;
  s.a_bx = (d.nyz / 2 + ang::kF2X - 1) / ang::kF2X;
  s.a_tiles = (long long)s.a_bx * (((long long)d.ncomp * d.ng * 2 + kBAngRep - 1) / kBAngRep);
  s.smem = std::max(sizeof(en::GroupPair) * (size_t)d.ng,
                    std::max((size_t)kBWarps * tr::kR * 32 * kBKV * sizeof(float),
                             sizeof(float2) * (size_t)d.nu * d.nv * ang::kF2X));
  return s;
}

bool batch_supported(int nu, int nv) { return nu <= 8 && nv <= 8 && angular_supported(nu, nv); }

cudaError_t launch_batch(const LaunchCtx &lc, int nu, int nv, const BatchBeam *beams, int nbeams,
                         const BatchTask *tasks, int ntasks, BatchQueue *q, unsigned long long *done,
                         unsigned long long *next, long long wait_cycles, size_t smem, double du, double dv) {
#define PBS_B(A, B)                                                                                              \
  if (nu == A && nv == B)                                                                                        \
    return go_batch<A, B>(lc, beams, nbeams, tasks, ntasks, q, done, next, wait_cycles, smem, du, dv);
  PBS_B(2, 2) PBS_B(4, 4) PBS_B(6, 6) PBS_B(8, 8) PBS_B(4, 8) PBS_B(8, 4) PBS_B(6, 4) PBS_B(4, 6)
#undef PBS_B
  return cudaErrorNotSupported;
}

}  // namespace pbs
